"""GPU parity: every call goes through the C ABI (libchfsi.so) and is compared
element by element with the FP64 CPU oracle on the same seeded inputs.

Tolerances:
* FP64 filter (CSR and BSR): relative Frobenius error <= 1e-12 (the target the
  method is held to; differences come from FMA contraction and summation order).
* Lanczos bounds: 1e-10 relative on a0 and b (and hence a).
* Ritz values: 1e-10 relative to max |theta| (CholQR2 vs Householder bases span
  the same space up to ~u cond(Y)).
* Adjoint: 1e-10 relative Frobenius on dX and dH against the oracle's reverse mode.
* Mixed precision: stated per variant below from the unit roundoff of the
  low-precision steps.
"""
import math

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
    assert torch.cuda.is_available()
    return P


DEV = "cuda"


def make_case(g, w, n, seed=1, s=0.1, core=0.0, orth=True):
    H = W.csr_grid(g, w, s, seed, core_frac=core, core_shift=2.0 if core else 0.0)
    X = W.start_block(H["N"], n, seed, orthonormalise=orth)
    return H, X


def bounds_for(oracle_mod, H, n, seed=1):
    v0 = W.lanczos_start(H["N"], seed)
    return oracle_mod.lanczos_bounds(H, v0, 20, n), v0


def to_dev(P, H):
    return P.CsrMatrix.from_arrays(H["row_ptr"], H["col"], H["val"], device=DEV)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV)


# --------------------------------------------------------------------------- filter FP64


@pytest.mark.parametrize("g,w,n,m", [
    (8, 2, 6, 1), (8, 2, 6, 2), (8, 3, 37, 10), (5, 1, 3, 7), (12, 3, 70, 13),
    (10, 2, 129, 5), (7, 3, 1, 9), (6, 4, 64, 20),
])
def test_filter_f64_csr_small(P, oracle_mod, g, w, n, m):
    H, X = make_case(g, w, n, seed=g * 10 + w)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, min(n, H["N"] // 4)))
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Y = P.filter(to_dev(P, H), dev(X), m, a, b, a0).cpu().numpy()
    assert rel_fro(Y, Yref) <= 1e-12


def test_filter_f64_odd_leading_dimensions(P, oracle_mod):
    """Row-major blocks with ld > n (views of wider buffers) and odd n."""
    H, X = make_case(8, 2, 9, seed=3)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 9)
    Yref = oracle_mod.filter(H, X, 6, a, b, a0)
    Xbig = torch.zeros((H["N"], 12), dtype=torch.float64, device=DEV)
    Xbig[:, :9] = dev(X)
    Ybig = torch.full((H["N"], 14), 7.0, dtype=torch.float64, device=DEV)
    P.filter(to_dev(P, H), Xbig[:, :9], 6, a, b, a0, out=Ybig[:, :9])
    assert rel_fro(Ybig[:, :9].cpu().numpy(), Yref) <= 1e-12
    assert torch.all(Ybig[:, 9:] == 7.0)          # padding untouched


def test_filter_f64_config_20cube_full(P, oracle_mod):
    """20^3 grid, w = 2, 64 states, m = 10: every output element."""
    wl = W.workload("g20_w2_n64_m10")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    Yref = oracle_mod.filter(H, X, wl.m, a, b, a0)
    Y = P.filter(to_dev(P, H), dev(X), wl.m, a, b, a0).cpu().numpy()
    assert rel_fro(Y, Yref) <= 1e-12


def test_filter_f64_config_40cube_sampled_columns(P, oracle_mod):
    """40^3 grid, w = 3, 1024 states, m = 20 at full size on the GPU (the bench
    launch); the oracle filters a seeded 48-column subset (columns are independent)."""
    wl = W.workload("g40_w3_n1024_m20")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    Y = P.filter(to_dev(P, H), dev(X), wl.m, a, b, a0).cpu().numpy()
    cols = W.column_subset(wl.n, 48, wl.seed)
    Yref = oracle_mod.filter(H, X[:, cols], wl.m, a, b, a0)
    assert rel_fro(Y[:, cols], Yref) <= 1e-12
    assert np.all(np.isfinite(Y))


def test_filter_determinism(P, oracle_mod):
    H, X = make_case(12, 3, 40, seed=5)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 40)
    Hd, Xd = to_dev(P, H), dev(X)
    Y1 = P.filter(Hd, Xd, 9, a, b, a0)
    Y2 = P.filter(Hd, Xd, 9, a, b, a0)
    assert torch.equal(Y1, Y2)


# --------------------------------------------------------------------------- filter BSR


def to_dev_bsr(P, B):
    return P.BsrMatrix.from_arrays(B["brow_ptr"], B["bcol"], B["val"], device=DEV)


@pytest.mark.parametrize("g,w,n,m", [(8, 2, 16, 4), (8, 3, 70, 9), (12, 4, 33, 6), (4, 1, 5, 3)])
def test_filter_f64_bsr(P, oracle_mod, g, w, n, m):
    H, X = make_case(g, w, n, seed=7 + g)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, min(n, H["N"] // 4)))
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Yb = P.filter(to_dev_bsr(P, B), dev(X[perm]), m, a, b, a0).cpu().numpy()
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    assert rel_fro(Y, Yref) <= 1e-12


# --------------------------------------------------------------------------- mixed precision


@pytest.mark.parametrize("low,tol", [("f32", 2e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("layout", ["csr", "bsr"])
def test_filter_mixed_schedule(P, oracle_mod, low, tol, layout):
    """L low-precision steps then FP64 steps.  The low steps carry relative
    rounding u_low (2^-24 for FP32, 2^-8 for BF16 operands) per step, amplified at
    most by the step count; the FP64 tail adds nothing measurable."""
    g, w, n, m, L = 8, 3, 24, 12, 8
    H, X = make_case(g, w, n, seed=21)
    (a, b, a0), _ = bounds_for(oracle_mod, H, n)
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    sched = P.mixed_schedule(m, L, low)
    if layout == "csr":
        Y = P.filter(to_dev(P, H), dev(X), m, a, b, a0, schedule=sched).cpu().numpy()
    else:
        B = W.bsr_from_csr(H, g)
        perm = B["perm"]
        Yb = P.filter(to_dev_bsr(P, B), dev(X[perm]), m, a, b, a0, schedule=sched).cpu().numpy()
        Y = np.empty_like(Yb)
        Y[perm] = Yb
    err = rel_fro(Y, Yref)
    assert err <= tol, err
    # all-low schedule widens the last FP32 iterate into Y
    if low == "f32" and layout == "csr":
        Yall = P.filter(to_dev(P, H), dev(X), m, a, b, a0, schedule=[low] * m).cpu().numpy()
        assert rel_fro(Yall, Yref) <= tol


@pytest.mark.parametrize("g,w,n,m,L", [(8, 3, 200, 9, 6), (12, 4, 128, 7, 7), (4, 1, 5, 4, 2), (8, 2, 64, 5, 5),
                                       (8, 2, 390, 5, 5)])
def test_bsr_tensor_core_bf16_matches_csr_bf16(P, oracle_mod, g, w, n, m, L):
    """tcgen05 BSR steps (BF16 operands, FP32 accumulation in TMEM) against the
    CUDA-core CSR steps with the same BF16 rounding of H and of Y_k: the two
    differ only in FP32 accumulation order (tolerance 20 u_fp32 per step, times
    the BF16 re-rounding it can flip), and both against the FP64 oracle."""
    H, X = make_case(g, w, n, seed=90 + g + n)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, min(n, H["N"] // 4)))
    sched = P.mixed_schedule(m, L, "bf16")
    Yc = P.filter(to_dev(P, H), dev(X), m, a, b, a0, schedule=sched).cpu().numpy()
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    ws = P.Workspace(DEV)
    Yb = P.filter(to_dev_bsr(P, B), dev(X[perm]), m, a, b, a0, schedule=sched, workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    assert np.all(np.isfinite(Y))
    assert rel_fro(Y, Yc) <= 2e-2
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    assert rel_fro(Y, Yref) <= 5e-2


@pytest.mark.parametrize("low", ["bf16", "f32"])
def test_hybrid_operator_mixed_schedule(P, oracle_mod, low):
    """CHFSI_HYBRID: BF16 prefix on the BSR blocks (tensor cores) or FP32 prefix on
    the blocked-order CSR, then the FP64 tail on the CSR; the backward pass and the
    bounds also accept the hybrid operator (they use its CSR)."""
    g, w, n, m, L = 8, 3, 70, 12, 8
    H, X = make_case(g, w, n, seed=23)
    (a, b, a0), v0 = bounds_for(oracle_mod, H, n)
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    Hp = W.permute_csr(H, perm)
    Hy = P.HybridMatrix(to_dev(P, Hp), to_dev_bsr(P, B))
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Yb = P.filter(Hy, dev(X[perm]), m, a, b, a0, schedule=P.mixed_schedule(m, L, low)).cpu().numpy()
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    assert rel_fro(Y, Yref) <= (5e-2 if low == "bf16" else 2e-5)
    Y64 = P.filter(Hy, dev(X[perm]), m, a, b, a0).cpu().numpy()
    Y[perm] = Y64
    assert rel_fro(Y, Yref) <= 1e-12
    a2, b2, a02 = P.lanczos_bounds(Hy, dev(v0[perm]), 20, n)
    assert abs(a02 - a0) <= 1e-9 * abs(a0) and abs(b2 - b) <= 1e-9 * abs(b)


@pytest.mark.parametrize("n", [136, 300, 520])
def test_bsr_tensor_core_single_step_exact_products(P, oracle_mod, n):
    """m = 1 with BF16-representable H and X: every product and every partial sum
    is exact in FP32, so the tensor-core step equals the oracle to FP32 rounding
    of the result -- for one span of states with a ragged second tile (136), and
    for several spans whose last one holds a single partial tile (300, 520)."""
    g, w = 8, 2
    H = W.csr_grid(g, w, 0.0, 3)
    H["val"] = np.round(H["val"] * 64) / 64             # few-bit values: exact in BF16
    Xr = np.random.default_rng(5).integers(-8, 9, size=(H["N"], n)) / 8.0
    a0, a, b = 1.0, 3.5, 14.0
    Yref = oracle_mod.filter(H, Xr, 1, a, b, a0)
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    Yb = P.filter(to_dev_bsr(P, B), dev(Xr[perm]), 1, a, b, a0, schedule=["bf16"]).cpu().numpy()
    Y = np.empty_like(Yb)
    Y[perm] = Yb
    assert rel_fro(Y, Yref) <= 1e-6


@pytest.mark.parametrize("g,w,n,m,L", [(8, 2, 6, 5, 5), (8, 3, 37, 10, 10), (12, 3, 70, 13, 9), (5, 1, 3, 7, 1),
                                       (10, 2, 129, 6, 6), (6, 4, 64, 20, 20), (8, 3, 301, 6, 6)])
def test_filter_f32x2_is_fp64_accurate(P, oracle_mod, g, w, n, m, L):
    """Two-float steps (hi + lo FP32 pairs, error-free transformations on the
    FP32 pipe) meet the FP64 filter tolerance against the FP64 oracle."""
    H, X = make_case(g, w, n, seed=g * 10 + w + 3)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, min(n, H["N"] // 4)))
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    ws = P.Workspace(DEV)
    Y = P.filter(to_dev(P, H), dev(X), m, a, b, a0, schedule=P.mixed_schedule(m, L, "f32x2"),
                 workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    assert rel_fro(Y, Yref) <= 1e-12


@pytest.mark.parametrize("schedule", [None, "f32x2"])
def test_unsorted_rows_with_duplicate_columns(P, oracle_mod, schedule):
    """Rows in random order with some entries split into two entries on the same
    column (CSR sums duplicates), on an odd row count: the FP64 step and the
    two-float row-pair step (whose merge of two rows must emit every entry once
    whatever the order) match the oracle on the sorted operator."""
    H, X = make_case(7, 2, 24, seed=57)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 24)
    rng = np.random.default_rng(5)
    rp, col, val = H["row_ptr"], H["col"], H["val"]
    rows_c, rows_v = [], []
    for r in range(H["N"]):
        c, v = col[rp[r]:rp[r + 1]].copy(), val[rp[r]:rp[r + 1]].copy()
        split = rng.random(len(c)) < 0.2
        frac = rng.random(int(split.sum()))
        c = np.concatenate([c, c[split]])
        v = np.concatenate([np.where(split, 0.0, v), v[split] * frac])
        v[np.flatnonzero(split)] = val[rp[r]:rp[r + 1]][split] * (1.0 - frac)
        order = rng.permutation(len(c))
        rows_c.append(c[order])
        rows_v.append(v[order])
    Hs = dict(N=H["N"], nnz=sum(len(c) for c in rows_c),
              row_ptr=np.concatenate([[0], np.cumsum([len(c) for c in rows_c])]).astype(np.int64),
              col=np.concatenate(rows_c).astype(np.int32), val=np.concatenate(rows_v))
    assert Hs["N"] % 2 == 1 and Hs["nnz"] > H["nnz"]
    m = 9
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    ws = P.Workspace(DEV)
    sched = None if schedule is None else [schedule] * m
    Y = P.filter(to_dev(P, Hs), dev(X), m, a, b, a0, schedule=sched, workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    assert rel_fro(Y, Yref) <= 1e-12


@pytest.mark.parametrize("schedule", [None, "f32", "f32x2", "bf16", "mixed"])
def test_column_slabs_and_views_of_wider_blocks(P, oracle_mod, schedule):
    """More than 512 states (the filter runs in column slabs of 512, here 512 + 512 +
    77 with an odd last slab) with X and Y column views of wider row-major blocks:
    results match the oracle and Y's columns beyond n are left untouched."""
    H, Xfull = make_case(8, 2, 1101, seed=61)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 64)
    m = 6
    n = Xfull.shape[1]
    Xw = torch.zeros((H["N"], 1210), dtype=torch.float64, device=DEV)
    Xw[:, :n] = dev(Xfull)
    Yw = torch.full((H["N"], 1306), 7.25, dtype=torch.float64, device=DEV)
    Xv, Yv = Xw[:, :n], Yw[:, :n]
    if schedule is None:
        sched = None
    elif schedule == "mixed":
        sched = P.mixed_schedule(m, 4, "f32x2")
    else:
        sched = [schedule] * m
    ws = P.Workspace(DEV)
    P.filter(to_dev(P, H), Xv, m, a, b, a0, schedule=sched, out=Yv, workspace=ws)
    assert P.read_status(ws) == 0
    Yref = oracle_mod.filter(H, Xfull, m, a, b, a0)
    tol = {"f32": 2e-5, "bf16": 5e-2}.get(schedule, 1e-12)
    assert rel_fro(Yv.cpu().numpy(), Yref) <= tol
    assert bool(torch.all(Yw[:, n:] == 7.25))


def _block_sparse_with_empty_block_row(seed=23):
    """A 256 x 256 symmetric operator of 64 x 64 dense blocks on a 4 x 4 block
    pattern whose block row (and column) 2 is empty: rows 128..191 hold no entry."""
    rng = np.random.default_rng(seed)
    pattern = np.array([[1, 1, 0, 1], [1, 1, 0, 0], [0, 0, 0, 0], [1, 0, 0, 1]], dtype=bool)
    A = np.zeros((256, 256))
    for I in range(4):
        for J in range(I, 4):
            if pattern[I, J]:
                blk = rng.standard_normal((64, 64)) * (0.05 if I != J else 0.1)
                if I == J:
                    blk = 0.5 * (blk + blk.T) + np.diag(np.linspace(1.0, 3.0, 64))
                A[64 * I:64 * I + 64, 64 * J:64 * J + 64] = blk
                A[64 * J:64 * J + 64, 64 * I:64 * I + 64] = blk.T
    brow_ptr, bcol, vals = [0], [], []
    for I in range(4):
        for J in range(4):
            if pattern[I, J]:
                bcol.append(J)
                vals.append(A[64 * I:64 * I + 64, 64 * J:64 * J + 64].copy())
        brow_ptr.append(len(bcol))
    B = dict(brow_ptr=np.array(brow_ptr, dtype=np.int32), bcol=np.array(bcol, dtype=np.int32),
             val=np.concatenate([v.ravel() for v in vals]))
    from tests.util import dense_to_csr
    return A, dense_to_csr(A, keep_zeros=False), B


@pytest.mark.parametrize("layout,schedule,tol", [("csr", None, 1e-12), ("csr", "f32x2", 1e-12), ("csr", "f32", 2e-5),
                                                 ("csr", "bf16", 5e-2), ("bsr", None, 1e-12), ("bsr", "bf16", 5e-2)])
def test_empty_rows_and_block_rows(P, oracle_mod, layout, schedule, tol):
    """Rows with no stored entry (and, in the blocked layout, a block row with no
    block, so its tensor-core accumulator is never written) filter to
    alpha (-c Y_k) - beta Y_{k-1}, as the oracle computes them."""
    A, H, B = _block_sparse_with_empty_block_row()
    assert np.all(np.diff(H["row_ptr"])[128:192] == 0)
    n, m = 40, 5
    X = np.linalg.qr(np.random.default_rng(3).standard_normal((256, n)))[0]
    lam = np.linalg.eigvalsh(A)          # 64 zero eigenvalues from the empty rows, then ~1..3.8
    a0, a, b = lam[0] - 0.01, lam[100], lam[-1] + 0.01
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Hd = to_dev(P, H) if layout == "csr" else to_dev_bsr(P, B)
    ws = P.Workspace(DEV)
    sched = None if schedule is None else [schedule] * m
    Y = P.filter(Hd, dev(X), m, a, b, a0, schedule=sched, workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    assert rel_fro(Y, Yref) <= tol


def _random_symmetric_csr(rng, N, density, long_rows=0, empty_rows=0):
    """Random symmetric sparse operator: a random pattern of the given density plus a
    diagonal, some rows made long (dense) and some emptied, values N(0, 1/nnz-row)."""
    A = (rng.random((N, N)) < density).astype(float) * rng.standard_normal((N, N))
    for r in rng.choice(N, size=long_rows, replace=False):
        A[r, :] = rng.standard_normal(N)
    A = np.triu(A) + np.triu(A, 1).T
    A += np.diag(rng.uniform(1.0, 3.0, N))
    for r in rng.choice(N, size=empty_rows, replace=False):
        A[r, :] = 0.0
        A[:, r] = 0.0
    A /= max(1.0, np.abs(A).sum(axis=1).max() / 4.0)
    from tests.util import dense_to_csr
    return A, dense_to_csr(A, keep_zeros=False)


@pytest.mark.parametrize("case", range(8))
def test_random_operators_all_precisions(P, oracle_mod, case):
    """Seeded random operators (random densities and sizes, a few dense rows that
    overflow the staged slice, a few empty rows, odd and even state counts) through
    every CSR arithmetic: FP64 and two-float to 1e-12, FP32 and BF16 operands to
    their rounding tolerances."""
    rng = np.random.default_rng(1000 + case)
    N = int(rng.integers(40, 700))
    A, H = _random_symmetric_csr(rng, N, float(rng.uniform(0.005, 0.1)), long_rows=int(rng.integers(0, 3)),
                                 empty_rows=int(rng.integers(0, 3)))
    n = int(rng.integers(1, 300))
    m = int(rng.integers(1, 12))
    X = rng.standard_normal((N, n)) / np.sqrt(N)
    lam = np.linalg.eigvalsh(A)
    a0, b = lam[0] - 0.05, lam[-1] + 0.05
    a = lam[0] + (lam[-1] - lam[0]) * float(rng.uniform(0.2, 0.6))
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Hd = to_dev(P, H)
    ws = P.Workspace(DEV)
    for sched, tol in ((None, 1e-12), ("f32x2", 1e-12), ("f32", 2e-5 * m), ("bf16", 5e-2)):
        s_ = None if sched is None else [sched] * m
        Y = P.filter(Hd, dev(X), m, a, b, a0, schedule=s_, workspace=ws).cpu().numpy()
        assert P.read_status(ws) == 0, sched
        assert rel_fro(Y, Yref) <= tol, (sched, N, n, m, rel_fro(Y, Yref))


@pytest.mark.parametrize("case", range(4))
def test_random_operators_closure_and_adjoint(P, oracle_mod, case):
    """Seeded random operators through the closure (CholQR2 + Rayleigh-Ritz, FP64 and
    two-float products) and the adjoint (FP64 and two-float sweeps) against the oracle."""
    rng = np.random.default_rng(2000 + case)
    N = int(rng.integers(80, 400))
    A, H = _random_symmetric_csr(rng, N, float(rng.uniform(0.01, 0.08)), long_rows=1, empty_rows=0)
    n = int(rng.integers(4, 60))
    m = int(rng.integers(2, 9))
    X = np.linalg.qr(rng.standard_normal((N, n)))[0]
    lam = np.linalg.eigvalsh(A)
    a0, b = lam[0] - 0.05, lam[-1] + 0.05
    a = lam[0] + (lam[-1] - lam[0]) * 0.4
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    Hd = to_dev(P, H)
    for prec in ("f64", "f32x2"):
        ritz, psi = P.rayleigh_ritz(Hd, dev(Y), cholqr_passes=2, precision=prec)
        _check_ritz(oracle_mod, H, Y, ritz.cpu().numpy(), psi.cpu().numpy(), orth_tol=1e-11)
    G = rng.standard_normal((N, n))
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    for prec in ("f64", "f32x2"):
        dX, dH = P.filter_backward(Hd, dev(X), dev(G), m, a, b, a0, precision=prec)
        assert rel_fro(dX.cpu().numpy(), dX_ref) <= 1e-10, prec
        assert rel_fro(dH.cpu().numpy(), dH_ref) <= 1e-10, prec


@pytest.mark.parametrize("case", range(4))
def test_random_block_operators_bsr_and_tensor_cores(P, oracle_mod, case):
    """Seeded random symmetric block patterns (odd and even block-row counts, empty
    block rows possible, unsorted block columns) of dense 64 x 64 blocks: the FP64 BSR
    step to 1e-12 and the tensor-core BF16 step (block-row pairs, zero block for a
    missing partner) to the BF16 tolerance, both against the oracle on the same H."""
    rng = np.random.default_rng(3000 + case)
    nbr = int(rng.integers(1, 10))
    pat = rng.random((nbr, nbr)) < float(rng.uniform(0.15, 0.6))
    pat = np.triu(pat) | np.triu(pat).T
    np.fill_diagonal(pat, rng.random(nbr) < 0.85)
    N = 64 * nbr
    A = np.zeros((N, N))
    for I in range(nbr):
        for J in range(I, nbr):
            if pat[I, J]:
                blk = rng.standard_normal((64, 64)) * 0.05
                if I == J:
                    blk = 0.5 * (blk + blk.T) + np.diag(rng.uniform(1.0, 3.0, 64))
                A[64 * I:64 * I + 64, 64 * J:64 * J + 64] = blk
                A[64 * J:64 * J + 64, 64 * I:64 * I + 64] = blk.T
    brow_ptr, bcol, vals = [0], [], []
    for I in range(nbr):
        cols = [J for J in range(nbr) if pat[I, J]]
        rng.shuffle(cols)
        for J in cols:
            bcol.append(J)
            vals.append(A[64 * I:64 * I + 64, 64 * J:64 * J + 64].copy())
        brow_ptr.append(len(bcol))
    if not bcol:
        pytest.skip("empty operator")
    B = dict(brow_ptr=np.array(brow_ptr, dtype=np.int32), bcol=np.array(bcol, dtype=np.int32),
             val=np.concatenate([v.ravel() for v in vals]))
    from tests.util import dense_to_csr
    H = dense_to_csr(A, keep_zeros=False)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(1, 8))
    X = rng.standard_normal((N, n)) / np.sqrt(N)
    lam = np.linalg.eigvalsh(A)
    a0, b = lam[0] - 0.05, lam[-1] + 0.05
    a = lam[0] + (lam[-1] - lam[0]) * 0.4
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    Bd = to_dev_bsr(P, B)
    ws = P.Workspace(DEV)
    for sched, tol in ((None, 1e-12), ("bf16", 5e-2)):
        s_ = None if sched is None else [sched] * m
        Y = P.filter(Bd, dev(X), m, a, b, a0, schedule=s_, workspace=ws).cpu().numpy()
        assert P.read_status(ws) == 0, sched
        assert rel_fro(Y, Yref) <= tol, (sched, nbr, n, m, rel_fro(Y, Yref))


@pytest.mark.parametrize("case", range(4))
def test_random_operators_lanczos_bounds(P, oracle_mod, case):
    """Seeded random operators (with empty rows: the spectrum then contains 0) through
    the GPU Lanczos bounds against the oracle's, and both bracket the spectrum."""
    rng = np.random.default_rng(4000 + case)
    N = int(rng.integers(60, 500))
    A, H = _random_symmetric_csr(rng, N, float(rng.uniform(0.01, 0.08)), long_rows=1,
                                 empty_rows=int(rng.integers(0, 3)))
    steps = int(rng.integers(5, 21))
    n_want = int(rng.integers(1, N // 4))
    v0 = rng.standard_normal(N)
    ra, rb, ra0 = oracle_mod.lanczos_bounds(H, v0, steps, n_want)
    a, b, a0 = P.lanczos_bounds(to_dev(P, H), dev(v0), steps, n_want)
    for x, y in ((a, ra), (b, rb), (a0, ra0)):
        assert abs(x - y) <= 1e-10 * max(1.0, abs(y))
    lam = np.linalg.eigvalsh(A)
    assert b >= lam[-1] - 1e-12 and a0 >= lam[0] - 1e-12 and a0 < a < b


def test_filter_f32x2_config_40cube_sampled_columns(P, oracle_mod):
    wl = W.workload("g40_w3_n1024_m20")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    Y = P.filter(to_dev(P, H), dev(X), wl.m, a, b, a0, schedule=["f32x2"] * wl.m).cpu().numpy()
    cols = W.column_subset(wl.n, 48, wl.seed)
    Yref = oracle_mod.filter(H, X[:, cols], wl.m, a, b, a0)
    assert rel_fro(Y[:, cols], Yref) <= 1e-12


# --------------------------------------------------------------------------- Lanczos


@pytest.mark.parametrize("g,w,n", [(8, 2, 32), (20, 2, 64), (12, 3, 100)])
def test_lanczos_bounds(P, oracle_mod, g, w, n):
    H, _ = make_case(g, w, 1, seed=31 + g)
    v0 = W.lanczos_start(H["N"], 5)
    a_r, b_r, a0_r = oracle_mod.lanczos_bounds(H, v0, 20, n)
    a, b, a0 = P.lanczos_bounds(to_dev(P, H), dev(v0), 20, n)
    for x, y in ((a, a_r), (b, b_r), (a0, a0_r)):
        assert abs(x - y) <= 1e-10 * abs(y)


def test_lanczos_tiny_breakdown(P, oracle_mod):
    """N < steps: the Krylov space fills up and the iteration stops with zero residual."""
    d = np.array([3.0, -1.0, 0.5, 7.25, 2.0, 4.5, -0.25, 6.0, 1.0, 5.5])
    N = d.size
    H = dict(N=N, nnz=N, row_ptr=np.arange(N + 1, dtype=np.int64), col=np.arange(N, dtype=np.int32), val=d)
    v0 = np.random.default_rng(2).standard_normal(N)
    a, b, a0 = P.lanczos_bounds(to_dev(P, H), dev(v0), 20, 2)
    assert abs(a0 - d.min()) < 1e-12 and abs(b - d.max()) < 1e-11


# --------------------------------------------------------------------------- Rayleigh-Ritz


def _check_ritz(oracle_mod, H, Y, ritz, psi, tol=1e-10, orth_tol=1e-12):
    theta, Psi_ref, _ = oracle_mod.rayleigh_ritz(H, Y)
    scale = np.max(np.abs(theta))
    assert np.max(np.abs(ritz - theta)) <= tol * scale
    n = Y.shape[1]
    assert np.max(np.abs(psi.T @ psi - np.eye(n))) <= orth_tol
    # Ritz vectors: compare projectors onto clusters of (numerically) equal values
    i = 0
    while i < n:
        j = i + 1
        while j < n and abs(theta[j] - theta[j - 1]) <= 1e-8 * scale:
            j += 1
        A, B = psi[:, i:j], Psi_ref[:, i:j]
        s = np.linalg.svd(A.T @ B, compute_uv=False)
        assert np.min(s) >= 1 - 1e-8, (i, j, s)
        i = j


@pytest.mark.parametrize("passes", [1, 2])
def test_rayleigh_ritz_small(P, oracle_mod, passes):
    H, X = make_case(8, 2, 20, seed=41)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 20)
    Y = oracle_mod.filter(H, X, 8, a, b, a0)
    ritz, psi = P.rayleigh_ritz(to_dev(P, H), dev(Y), cholqr_passes=passes)
    _check_ritz(oracle_mod, H, Y, ritz.cpu().numpy(), psi.cpu().numpy())


def test_rayleigh_ritz_full_space_is_eigh(P, oracle_mod):
    H, _ = make_case(6, 2, 1, seed=43)
    N = H["N"]
    Y = np.linalg.qr(np.random.default_rng(3).standard_normal((N, N)))[0]
    ritz, psi = P.rayleigh_ritz(to_dev(P, H), dev(Y))
    from tests.util import csr_to_dense
    lam = np.linalg.eigvalsh(csr_to_dense(H))
    assert np.max(np.abs(ritz.cpu().numpy() - lam)) <= 1e-12 * np.max(np.abs(lam))


def test_rayleigh_ritz_config_40cube(P, oracle_mod):
    """Full 40^3 / 1024-state cycle: filter (m = 20) then CholQR2 + RR on the GPU;
    the oracle runs its own filter and Householder/LAPACK closure on the same inputs."""
    wl = W.workload("g40_w3_n1024_m20")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    Hd = to_dev(P, H)
    Yd = P.filter(Hd, dev(X), wl.m, a, b, a0)
    ritz, psi = P.rayleigh_ritz(Hd, Yd, cholqr_passes=2)
    Yref = oracle_mod.filter(H, X, wl.m, a, b, a0)
    theta, _, _ = oracle_mod.rayleigh_ritz(H, Yref)
    assert np.max(np.abs(ritz.cpu().numpy() - theta)) <= 1e-10 * np.max(np.abs(theta))


@pytest.mark.parametrize("passes", [1, 2])
def test_rayleigh_ritz_f32x2_products(P, oracle_mod, passes):
    """Two-float Gram / projection / rotation products (FP64 Cholesky and
    eigensolve): Ritz values and vectors at the FP64 closure's tolerances."""
    H, X = make_case(8, 2, 20, seed=45)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 20)
    Y = oracle_mod.filter(H, X, 8, a, b, a0)
    ritz, psi = P.rayleigh_ritz(to_dev(P, H), dev(Y), cholqr_passes=passes, precision="f32x2")
    # one CholQR pass leaves ~u cond(Y)^2 loss of orthogonality, with the two-float
    # unit roundoff u = 2^-48 (cond(Y) ~ 30 here); the second pass restores ~u
    _check_ritz(oracle_mod, H, Y, ritz.cpu().numpy(), psi.cpu().numpy(),
                orth_tol=1e-12 if passes == 2 else 1e-10)


def test_rayleigh_ritz_f32x2_config_40cube(P, oracle_mod):
    wl = W.workload("g40_w3_n1024_m20")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    Hd = to_dev(P, H)
    Yd = P.filter(Hd, dev(X), wl.m, a, b, a0, schedule=["f32x2"] * wl.m)
    ritz, psi = P.rayleigh_ritz(Hd, Yd, cholqr_passes=2, precision="f32x2")
    Yref = oracle_mod.filter(H, X, wl.m, a, b, a0)
    theta, _, _ = oracle_mod.rayleigh_ritz(H, Yref)
    assert np.max(np.abs(ritz.cpu().numpy() - theta)) <= 1e-10 * np.max(np.abs(theta))
    p = psi.cpu().numpy()
    assert np.max(np.abs(p.T @ p - np.eye(wl.n))) <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32x2", "ozaki"])
def test_rayleigh_ritz_blocked_triangular_inverse(P, oracle_mod, precision):
    """2100 states: R^-1 of CholQR is formed by halves (1088 + 1012, the first half again
    by halves 576 + 512), the off-diagonal blocks by products (Ozaki products in the
    Ozaki closure) -- Ritz values and vectors at the FP64 closure's tolerances."""
    H, X = make_case(20, 2, 2100, seed=47)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 2100, 47)
    Y = oracle_mod.filter(H, X, 6, a, b, a0)
    ritz, psi = P.rayleigh_ritz(to_dev(P, H), dev(Y), cholqr_passes=2, precision=precision)
    _check_ritz(oracle_mod, H, Y, ritz.cpu().numpy(), psi.cpu().numpy())


def test_rayleigh_ritz_rank_deficient_reports_cholesky(P, oracle_mod):
    H, X = make_case(6, 2, 8, seed=44)
    X[:, 3] = 0.0
    with pytest.raises(P.ChfsiError) as e:
        P.rayleigh_ritz(to_dev(P, H), dev(X), cholqr_passes=1)
    assert e.value.code == 4


@pytest.mark.parametrize("rr_precision,schedule", [("f64", None), ("f32x2", "f32x2")])
def test_repeated_cycles_converge_to_eigh(P, oracle_mod, rr_precision, schedule):
    """Several ChFSI cycles (Psi of one cycle is X of the next, Zhou-Saad bound
    updates): the lowest 36 of 48 Ritz values converge to brute-force eigvalsh."""
    from tests.util import csr_to_dense
    g, w, n, m = 10, 2, 48, 10
    H = W.csr_grid(g, w, 0.1, 7)
    lam = np.linalg.eigvalsh(csr_to_dense(H))
    X = W.start_block(H["N"], n, 7)
    sched = None if schedule is None else [schedule] * m
    ritz, psi, hist = P.solve(to_dev(P, H), dev(X), m, 9, dev(W.lanczos_start(H["N"], 7)), schedule=sched,
                              rr_precision=rr_precision)
    th = ritz.cpu().numpy()
    assert np.max(np.abs(th[:36] - lam[:36]) / np.abs(lam[:36])) <= 1e-12
    errs = [np.max(np.abs(h.cpu().numpy()[:36] - lam[:36])) for h in hist]
    assert errs[0] > 1e-3 and errs[-1] < 1e-11          # it did converge, from far away
    p = psi.cpu().numpy()
    A = csr_to_dense(H)
    assert np.max(np.abs(p.T @ p - np.eye(n))) <= 1e-12
    r = A @ p[:, :36] - p[:, :36] * th[:36]
    assert np.max(np.linalg.norm(r, axis=0)) <= 1e-6


# --------------------------------------------------------------------------- adjoint


@pytest.mark.parametrize("g,w,n,m,stride", [(8, 2, 5, 7, 0), (6, 3, 4, 9, 2), (8, 2, 6, 16, 1), (5, 1, 3, 4, 9)])
def test_adjoint_matches_oracle(P, oracle_mod, g, w, n, m, stride):
    H, X = make_case(g, w, n, seed=50 + m)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, n))
    wts = W.loss_weights(H["N"], 3)
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    G = 2.0 * wts[:, None] * Y
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    dX, dH = P.filter_backward(to_dev(P, H), dev(X), dev(G), m, a, b, a0, ckpt_stride=stride)
    assert rel_fro(dX.cpu().numpy(), dX_ref) <= 1e-10
    assert rel_fro(dH.cpu().numpy(), dH_ref) <= 1e-10


@pytest.mark.parametrize("g,w,n,m,stride", [(8, 2, 5, 7, 0), (6, 3, 4, 9, 2), (8, 2, 6, 16, 1), (10, 2, 70, 6, 0)])
def test_adjoint_f32x2_matches_oracle(P, oracle_mod, g, w, n, m, stride):
    """Two-float reverse sweep (replay, reverse recurrence, dH products) against the
    oracle's FP64 reverse mode at the adjoint tolerance."""
    H, X = make_case(g, w, n, seed=80 + m)
    (a, b, a0), _ = bounds_for(oracle_mod, H, max(1, n))
    wts = W.loss_weights(H["N"], 3)
    G = 2.0 * wts[:, None] * oracle_mod.filter(H, X, m, a, b, a0)
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    dX, dH = P.filter_backward(to_dev(P, H), dev(X), dev(G), m, a, b, a0, ckpt_stride=stride, precision="f32x2")
    assert rel_fro(dX.cpu().numpy(), dX_ref) <= 1e-10
    assert rel_fro(dH.cpu().numpy(), dH_ref) <= 1e-10


@pytest.mark.parametrize("precision", ["f64", "f32x2"])
def test_adjoint_column_slabs_and_views(P, oracle_mod, precision):
    """More than 512 states: the reverse sweep runs in column slabs (512 + 512 + 7),
    each slab adding its part of dH; X and dY are column views of wider blocks."""
    H, Xfull = make_case(6, 2, 1031, seed=67)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 32)
    m = 7
    n = Xfull.shape[1]
    wts = W.loss_weights(H["N"], 5)
    G = 2.0 * wts[:, None] * oracle_mod.filter(H, Xfull, m, a, b, a0)
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, Xfull, m, a, b, a0, G)
    Xw = torch.zeros((H["N"], 1100), dtype=torch.float64, device=DEV)
    Gw = torch.zeros((H["N"], 1042), dtype=torch.float64, device=DEV)
    Xw[:, :n] = dev(Xfull)
    Gw[:, :n] = dev(G)
    dX, dH = P.filter_backward(to_dev(P, H), Xw[:, :n], Gw[:, :n], m, a, b, a0, precision=precision)
    assert rel_fro(dX.cpu().numpy(), dX_ref) <= 1e-10
    assert rel_fro(dH.cpu().numpy(), dH_ref) <= 1e-10


def test_adjoint_autograd_and_finite_differences(P, oracle_mod):
    """L = tr(Y^T W Y) through torch.autograd; dL/dH checked against central
    differences (step 1e-6) of the GPU forward on sampled entries."""
    H, X = make_case(8, 2, 6, seed=61)
    m = 10
    (a, b, a0), _ = bounds_for(oracle_mod, H, 6)
    wts = dev(W.loss_weights(H["N"], 4))
    Hd = to_dev(P, H)
    Xd = dev(X).requires_grad_(True)
    hv = Hd.val.clone().requires_grad_(True)
    Y = P.ChebyshevFilter.apply(Xd, hv, Hd, m, a, b, a0)
    L = (wts[:, None] * Y * Y).sum()
    L.backward()
    G = 2.0 * W.loss_weights(H["N"], 4)[:, None] * oracle_mod.filter(H, X, m, a, b, a0)
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    assert rel_fro(Xd.grad.cpu().numpy(), dX_ref) <= 1e-10
    assert rel_fro(hv.grad.cpu().numpy(), dH_ref) <= 1e-10

    def loss(val):
        Hp = P.CsrMatrix(Hd.row_ptr, Hd.col, val, Hd.n_rows)
        Yp = P.filter(Hp, dev(X), m, a, b, a0)
        return math.fsum(((wts[:, None] * Yp * Yp).sum(dim=1)).cpu().numpy())

    scale = float(hv.grad.abs().max())
    step = 1e-6
    for p in np.random.default_rng(0).choice(H["nnz"], 12, replace=False):
        vp, vm = Hd.val.clone(), Hd.val.clone()
        vp[p] += step
        vm[p] -= step
        fd = (loss(vp) - loss(vm)) / (2 * step)
        assert abs(fd - float(hv.grad[p])) <= 1e-6 * scale


def test_adjoint_config_32cube(P, oracle_mod):
    """32^3 grid, w = 2, 512 states, m = 16: GPU backward with sqrt(m)
    checkpointing at full size against the oracle's stored-iterate reverse mode."""
    wl = W.workload("g32_w2_n512_m16")
    H, X = make_case(wl.g, wl.w, wl.n, seed=wl.seed)
    (a, b, a0), _ = bounds_for(oracle_mod, H, wl.n, wl.seed)
    wts = W.loss_weights(H["N"], wl.seed)
    Hd = to_dev(P, H)
    Yd = P.filter(Hd, dev(X), wl.m, a, b, a0)
    Gd = 2.0 * dev(wts)[:, None] * Yd
    dX, dH = P.filter_backward(Hd, dev(X), Gd, wl.m, a, b, a0)
    G = Gd.cpu().numpy()
    dX_ref, dH_ref = oracle_mod.filter_adjoint(H, X, wl.m, a, b, a0, G)
    assert rel_fro(dX.cpu().numpy(), dX_ref) <= 1e-10
    assert rel_fro(dH.cpu().numpy(), dH_ref) <= 1e-10


def test_checkpoint_replay_is_bitwise(P, oracle_mod):
    """Different checkpoint strides replay the same forward kernels: identical results."""
    H, X = make_case(8, 2, 6, seed=71)
    m = 12
    (a, b, a0), _ = bounds_for(oracle_mod, H, 6)
    G = dev(np.random.default_rng(1).standard_normal(X.shape))
    Hd, Xd = to_dev(P, H), dev(X)
    outs = [P.filter_backward(Hd, Xd, G, m, a, b, a0, ckpt_stride=s) for s in (1, 3, 4, 12)]
    for dX, dH in outs[1:]:
        assert torch.equal(dX, outs[0][0]) and torch.equal(dH, outs[0][1])


# --------------------------------------------------------------------------- error paths


def test_error_paths(P, oracle_mod):
    H, X = make_case(6, 2, 4, seed=81)
    Hd, Xd = to_dev(P, H), dev(X)
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Hd, Xd, 5, 1.0, 2.0, 1.5)                 # a0 inside [a, b]
    assert e.value.code == 2
    # a column index out of range: the kernel skips it and reports PATTERN
    bad = dict(H)
    bad["col"] = H["col"].copy()
    bad["col"][17] = H["N"] + 5
    ws = P.Workspace(DEV)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 4)
    P.filter(to_dev(P, bad), Xd, 3, a, b, a0, workspace=ws)
    assert P.read_status(ws) == 3
    # NaN input is reported as non-finite
    Xn = Xd.clone()
    Xn[3, 1] = float("nan")
    P.filter(Hd, Xn, 3, a, b, a0, workspace=ws)
    assert P.read_status(ws) == 5
    # a clean call leaves the status word clear
    P.filter(Hd, Xd, 3, a, b, a0, workspace=ws)
    assert P.read_status(ws) == 0


def test_edge_cases_empty_and_unsupported(P, oracle_mod):
    """n_cols = 0 is a no-op; two-float needs the CSR layout; a schedule must list
    the low-precision steps as a prefix; single-row operators work."""
    import ctypes
    from paper_2110_15853_gb300 import _abi
    lib = P.load()
    H, X = make_case(4, 1, 3, seed=99)
    Hd = to_dev(P, H)
    desc = Hd.descriptor()
    ws = P.Workspace(DEV).get(1 << 20)
    Xd = dev(X)
    Y = torch.full_like(Xd, 3.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.chfsi_filter(ctypes.byref(desc), Xd.data_ptr(), 3, Y.data_ptr(), 3, 0, 4, 1.0, 2.0, 0.0, None,
                          ws.data_ptr(), ws.numel(), stream)
    assert rc == 0 and torch.all(Y == 3.0)
    B = W.bsr_from_csr(H, 4)
    Bd = to_dev_bsr(P, B)
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Bd, dev(X[B["perm"]]), 4, 1.0, 2.0, 0.0, schedule=["f32x2"] * 4)
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED
    with pytest.raises(P.ChfsiError) as e:
        P.rayleigh_ritz(Bd, dev(X[B["perm"]]), precision="f32x2")
    assert e.value.code == _abi.CHFSI_ERR_UNSUPPORTED
    with pytest.raises(P.ChfsiError) as e:
        P.filter(Hd, Xd, 4, 1.0, 2.0, 0.0, schedule=["f64", "f32", "f64", "f64"])
    assert e.value.code == _abi.CHFSI_ERR_ARG
    # a 1 x 1 operator: the filter is the scalar T_m((h - c)/e) / T_m(tau)
    one = dict(N=1, nnz=1, row_ptr=np.array([0, 1], dtype=np.int64), col=np.array([0], dtype=np.int32),
               val=np.array([0.3]))
    x = np.array([[1.5, -2.0]])
    y = P.filter(to_dev(P, one), dev(x), 7, 1.0, 2.0, 0.0).cpu().numpy()
    assert rel_fro(y, oracle_mod.filter(one, x, 7, 1.0, 2.0, 0.0)) <= 1e-14


@pytest.mark.parametrize("schedule", [None, "f32x2", "f32"])
def test_long_rows_use_the_unstaged_path(P, oracle_mod, schedule):
    """Rows too long for the CTA's shared-memory slice (a dense 1000 x 1000
    symmetric H: 8 rows x 1000 entries > the staging capacity) read their entries
    from global memory instead; results are unchanged."""
    from tests.util import dense_to_csr
    rng = np.random.default_rng(17)
    N, n, m = 1000, 16, 5
    A = rng.standard_normal((N, N)) * 0.01
    A = 0.5 * (A + A.T) + np.diag(np.linspace(1.0, 3.0, N))
    H = dense_to_csr(A)
    X = np.linalg.qr(rng.standard_normal((N, n)))[0]
    lam = np.linalg.eigvalsh(A)
    a0, a, b = lam[0] - 0.01, lam[40], lam[-1] + 0.01
    Yref = oracle_mod.filter(H, X, m, a, b, a0)
    ws = P.Workspace(DEV)
    sched = None if schedule is None else [schedule] * m
    Y = P.filter(to_dev(P, H), dev(X), m, a, b, a0, schedule=sched, workspace=ws).cpu().numpy()
    assert P.read_status(ws) == 0
    assert rel_fro(Y, Yref) <= (2e-5 if schedule == "f32" else 1e-12)


def test_nonfinite_reported_by_every_arithmetic(P, oracle_mod):
    H, X = make_case(6, 2, 8, seed=81)
    (a, b, a0), _ = bounds_for(oracle_mod, H, 8)
    Xn = dev(X)
    Xn[5, 3] = float("inf")
    ws = P.Workspace(DEV)
    for sched in (None, ["f32x2"] * 3, ["f32"] * 3, ["bf16"] * 3):
        P.filter(to_dev(P, H), Xn, 3, a, b, a0, schedule=sched, workspace=ws)
        assert P.read_status(ws) == 5, sched
