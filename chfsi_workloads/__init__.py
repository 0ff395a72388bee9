"""Seeded synthetic inputs for the ChFSI filter (shared by the oracle and the CUDA path).

This module holds only input data: the sparse symmetric Hamiltonian H on a 3-D
tensor-index grid, its blocked (BSR) re-ordering, the wavefunction block X, the
Lanczos start vector and the loss weights.  It contains none of the filter's
arithmetic (no Chebyshev coefficients, no SpMM, no orthonormalisation method of
the solver), so that the oracle and the GPU path can both take their inputs from
here without sharing any of the method.

Stand-in for the paper's Hamiltonians.  The paper's H^L (projection of the
Kohn-Sham operator on an L1-localised Tucker basis, Sec. 3.3, Eq. "KS-Hamiltonian
projection") is sparse, symmetric, dense near the diagonal and sparser away from
it (Sec. 4.1), and comes from a separable operator H1+H2+H3 (Sec. 3.2.1).  The
Al/Si matrices are not available, so H is generated as:

* composite index I = (i1*g + i2)*g + i3 with i3 fastest (Sec. 3.2.3: T_K with
  K = (r1, r2, r3));
* pattern: every (I, J) with |i_d - j_d| <= w in all three directions, clipped at
  the grid edge (every pattern entry is stored, even if its value is tiny);
* kinetic part A (x) I (x) I + I (x) A (x) I + I (x) I (x) A with the 1-D banded
  SPD matrix A: diagonal 2.5, off-diagonal -1/(1+|d|)^2 for 1 <= |d| <= w;
* potential V_IJ = V_JI = s * z * exp(-(d1^2 + d2^2 + d3^2)), z ~ N(0, 1) drawn
  once per unordered pair and mirrored;
* optionally a fraction of rows with a +-shift on the diagonal (atomic cores).

Random numbers come from numpy's Philox counter-based generator (Salmon et al.,
SC'11), keyed by (seed, stream id), so every array can be regenerated anywhere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "workload", "offsets", "csr_grid", "blocked_permutation",
    "bsr_from_csr", "gaussian", "start_block", "lanczos_start", "loss_weights",
    "row_subset", "column_subset", "permute_csr", "banded_operator", "split_from_csr",
]

SEED_BASE = 2110158530

# stream ids for the Philox keys
_STREAM_POTENTIAL = 100      # + offset index
_STREAM_CORES = 50
_STREAM_X = 1000
_STREAM_V0 = 1001
_STREAM_W = 1002
_STREAM_SUBSET = 1003
_STREAM_BAND = 2000
_STREAM_FAR = 2001


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic filter workload: grid edge g, band w, n columns, degree m."""
    name: str
    g: int
    w: int
    n: int
    m: int
    s: float
    seed: int
    core_frac: float = 0.0
    core_shift: float = 0.0
    low_steps: int = 0          # leading low-precision steps of the mixed schedule

    @property
    def N(self) -> int:
        return self.g ** 3


WORKLOADS = {
    # plain FP64 filter, degree 10, 20^3 grid, w=2, 64 states
    "g20_w2_n64_m10": Workload("g20_w2_n64_m10", 20, 2, 64, 10, 0.1, SEED_BASE + 1),
    # mid-scale FP64 filter + one CholQR / Rayleigh-Ritz cycle, 40^3 grid, w=3, 1024 states
    "g40_w3_n1024_m20": Workload("g40_w3_n1024_m20", 40, 3, 1024, 20, 0.1, SEED_BASE + 2),
    # mixed precision: 20 low-precision steps then 4 FP64 steps, 48^3 grid, 4096 states
    "g48_w3_n4096_m24": Workload("g48_w3_n4096_m24", 48, 3, 4096, 24, 0.1, SEED_BASE + 3,
                                 low_steps=20),
    # adjoint: 32^3 grid, w=2, 512 states, degree 16
    "g32_w2_n512_m16": Workload("g32_w2_n512_m16", 32, 2, 512, 16, 0.1, SEED_BASE + 4),
    # large: 64^3 grid, w=4, 6000 states, degree 30, amplitude 0.3, 5% core rows +-2.0
    "g64_w4_n6000_m30": Workload("g64_w4_n6000_m30", 64, 4, 6000, 30, 0.3, SEED_BASE + 5,
                                 core_frac=0.05, core_shift=2.0),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def offsets(w: int) -> np.ndarray:
    """All (d1, d2, d3) in [-w, w]^3 in lexicographic order; shape (K, 3)."""
    r = np.arange(-w, w + 1)
    d1, d2, d3 = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([d1.ravel(), d2.ravel(), d3.ravel()], axis=1)


def _kinetic_1d(d: int) -> float:
    return 2.5 if d == 0 else -1.0 / (1.0 + abs(d)) ** 2


def csr_grid(g: int, w: int, s: float, seed: int, core_frac: float = 0.0,
             core_shift: float = 0.0) -> dict:
    """Kronecker-banded symmetric H on a g^3 grid in CSR (columns ascending per row).

    Returns dict(N, nnz, row_ptr[int64, N+1], col[int32, nnz], val[float64, nnz]).
    """
    N = g ** 3
    offs = offsets(w)
    K = offs.shape[0]
    center = K // 2
    idx = np.arange(N, dtype=np.int64)
    i1, i2, i3 = idx // (g * g), (idx // g) % g, idx % g
    lin = offs[:, 0] * g * g + offs[:, 1] * g + offs[:, 2]

    vals = np.zeros((K, N), dtype=np.float64)
    mask = np.zeros((K, N), dtype=bool)
    for k in range(K):
        d1, d2, d3 = (int(x) for x in offs[k])
        valid = ((i1 + d1 >= 0) & (i1 + d1 < g) & (i2 + d2 >= 0) & (i2 + d2 < g)
                 & (i3 + d3 >= 0) & (i3 + d3 < g))
        mask[k] = valid
        nz = (d1 != 0) + (d2 != 0) + (d3 != 0)
        kin = 0.0
        if nz == 0:
            kin = 3 * _kinetic_1d(0)
        elif nz == 1:
            kin = _kinetic_1d(d1 + d2 + d3)
        damp = s * math.exp(-(d1 * d1 + d2 * d2 + d3 * d3))
        ku = k if k >= center else K - 1 - k          # the upper offset of the pair
        z = _rng(seed, _STREAM_POTENTIAL + ku).standard_normal(N)
        if k < center:
            # entry (I, I - o) mirrors (I - o, I), whose draw sits at row I - o
            z = np.roll(z, int(lin[ku]))               # z[I - o] at position I (valid I only)
        vals[k] = np.where(valid, kin + damp * z, 0.0)

    if core_frac > 0.0:
        r = _rng(seed, _STREAM_CORES)
        pick = r.random(N) < core_frac
        sign = np.where(r.random(N) < 0.5, -1.0, 1.0)
        vals[center] += np.where(pick, sign * core_shift, 0.0)

    maskT = mask.T
    counts = maskT.sum(axis=1)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cols = (idx[:, None] + lin[None, :])[maskT].astype(np.int32)
    val = vals.T[maskT].copy()
    del vals, mask, maskT
    return dict(N=N, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=cols, val=val)


def blocked_permutation(g: int, bs: int = 4) -> np.ndarray:
    """perm[r_new] = r_old for the block-major ordering of bs^3 sub-cubes.

    New index = B * bs^3 + ((l1 * bs) + l2) * bs + l3 with block index
    B = (b1 * (g/bs) + b2) * (g/bs) + b3 and i_d = b_d * bs + l_d.
    """
    if g % bs:
        raise ValueError("grid edge must be a multiple of the block edge")
    G = g // bs
    r = np.arange(g ** 3, dtype=np.int64)
    B, loc = r // bs ** 3, r % bs ** 3
    b1, b2, b3 = B // (G * G), (B // G) % G, B % G
    l1, l2, l3 = loc // (bs * bs), (loc // bs) % bs, loc % bs
    i1, i2, i3 = b1 * bs + l1, b2 * bs + l2, b3 * bs + l3
    return (i1 * g + i2) * g + i3


def bsr_from_csr(csr: dict, g: int, bs: int = 4) -> dict:
    """Blocked-CSR copy of H in block-major order (pure data movement).

    Returns dict(perm, n_block_rows, n_blocks, bdim, brow_ptr[int32], bcol[int32],
    val[float64, n_blocks*bdim*bdim] row-major per block).  Row r of the blocked
    matrix is row perm[r] of H; X and Y are permuted with the same perm.
    """
    N = csr["N"]
    bdim = bs ** 3
    perm = blocked_permutation(g, bs)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N, dtype=np.int64)
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(csr["row_ptr"]))
    r_new = inv[rows]
    c_new = inv[csr["col"].astype(np.int64)]
    br, bc = r_new // bdim, c_new // bdim
    nbr = N // bdim
    key = br * nbr + bc
    ukeys, block_of = np.unique(key, return_inverse=True)
    nblocks = ukeys.shape[0]
    ub_r, ub_c = ukeys // nbr, ukeys % nbr
    brow_ptr = np.zeros(nbr + 1, dtype=np.int64)
    np.cumsum(np.bincount(ub_r, minlength=nbr), out=brow_ptr[1:])
    val = np.zeros(nblocks * bdim * bdim, dtype=np.float64)
    val[block_of * bdim * bdim + (r_new % bdim) * bdim + (c_new % bdim)] = csr["val"]
    return dict(perm=perm, n_block_rows=nbr, n_blocks=int(nblocks), bdim=bdim,
                brow_ptr=brow_ptr.astype(np.int32), bcol=ub_c.astype(np.int32), val=val)


def permute_csr(csr: dict, perm: np.ndarray) -> dict:
    """CSR of P H P^T: row r of the result is row perm[r] of H, columns renumbered
    to the new order and sorted ascending (pure data movement)."""
    N = csr["N"]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N, dtype=np.int64)
    counts = np.diff(csr["row_ptr"])[perm]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    starts = csr["row_ptr"][perm]
    idx = np.repeat(starts - row_ptr[:-1], counts) + np.arange(row_ptr[-1], dtype=np.int64)
    cols = inv[csr["col"][idx].astype(np.int64)]
    vals = csr["val"][idx]
    rows = np.repeat(np.arange(N, dtype=np.int64), counts)
    order = np.lexsort((cols, rows))
    return dict(N=N, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=cols[order].astype(np.int32),
                val=vals[order].copy())


def gaussian(shape, seed: int, stream: int) -> np.ndarray:
    return _rng(seed, stream).standard_normal(shape)


def start_block(N: int, n: int, seed: int, orthonormalise: bool | None = None,
                out: np.ndarray | None = None) -> np.ndarray:
    """X: N x n Gaussian, orthonormalised by LAPACK Householder QR when affordable.

    For N*n^2 above 2e11 (the 48^3 and 64^3 workloads) a host QR takes too long,
    and X is the Gaussian block scaled by 1/sqrt(N) (columns nearly orthonormal);
    that block can be written into `out` (a C-contiguous float64 N x n array, e.g.
    the numpy view of pinned host memory), drawn in row chunks from the same
    Philox stream so that the values do not depend on the chunking.
    """
    if orthonormalise is None:
        orthonormalise = N * n * n <= 2e11
    if orthonormalise:
        X, _ = np.linalg.qr(gaussian((N, n), seed, _STREAM_X))
        X = np.ascontiguousarray(X)
        if out is not None:
            out[...] = X
            return out
        return X
    if out is None:
        out = np.empty((N, n), dtype=np.float64)
    if out.shape != (N, n) or out.dtype != np.float64 or not out.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 (N, n) array")
    rng = _rng(seed, _STREAM_X)
    root = math.sqrt(N)
    rows = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, N, rows):
        blk = out[r0:r0 + rows]
        rng.standard_normal(out=blk)
        blk /= root
    return out


def lanczos_start(N: int, seed: int) -> np.ndarray:
    """Lanczos start vector (unnormalised Gaussian)."""
    return gaussian(N, seed, _STREAM_V0)


def loss_weights(N: int, seed: int) -> np.ndarray:
    """Diagonal W of the loss L = tr(Y^T W Y), W_ii ~ N(0, 1)."""
    return gaussian(N, seed, _STREAM_W)


def row_subset(N: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted row indices (for sampled checks at full size)."""
    return np.sort(_rng(seed, _STREAM_SUBSET).permutation(N)[:k])


def column_subset(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted column indices (column independence of the filter)."""
    return np.sort(_rng(seed, _STREAM_SUBSET + 1).permutation(n)[:k])


def banded_operator(N: int, band: int, far: int, s: float, seed: int) -> dict:
    """Symmetric H whose density decays away from the diagonal, in CSR (columns
    ascending): every (i, j) with |i - j| <= band is stored (dense near the diagonal),
    with H_ij = H_ji = exp(-|i - j| / (band / 4)) (-0.5 + s z_ij) off the diagonal and
    H_ii = 2.5 + s z_ii; outside the band about `far` random couplings per row (pairs
    drawn uniformly with |i - j| > band, value 0.01 z, mirrored) -- a stand-in for the
    paper's H^L, whose diagonal blocks are much denser than the rest (Sec. 4.1).
    """
    rng = _rng(seed, _STREAM_BAND)
    d = np.arange(-band, band + 1)
    i = np.repeat(np.arange(N, dtype=np.int64), d.size)
    j = i + np.tile(d, N)
    keep = (j >= 0) & (j < N)
    i, j = i[keep], j[keep]
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    # one draw per unordered pair, keyed by (lo, offset) so that (i, j) and (j, i) agree
    zz = rng.standard_normal((N, band + 1))
    z = zz[lo, hi - lo]
    off = np.abs(i - j)
    val = np.where(off == 0, 2.5 + s * z, np.exp(-off / (band / 4.0)) * (-0.5 + s * z))
    # far couplings
    r2 = _rng(seed, _STREAM_FAR)
    cnt = N * far // 2
    a = r2.integers(0, N, size=cnt)
    b = r2.integers(0, N, size=cnt)
    ok = np.abs(a - b) > band
    a, b = a[ok], b[ok]
    pair = np.unique(np.minimum(a, b) * N + np.maximum(a, b))
    fa, fb = pair // N, pair % N
    fz = 0.01 * r2.standard_normal(pair.size)
    rows = np.concatenate([i, fa, fb])
    cols = np.concatenate([j, fb, fa])
    vals = np.concatenate([val, fz, fz])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=N), out=row_ptr[1:])
    return dict(N=N, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=cols.astype(np.int32), val=vals.copy())


def split_from_csr(csr: dict, block: int) -> dict:
    """The split storage of H (pure data movement): rows in blocks of `block`; the
    entries whose column lies in the row's own block go to a dense block x block
    diagonal block (stacked, zero-padded past N), the rest to an off-diagonal CSR in
    stored order.  Returns dict(block, n_blocks, diag[float64, n_blocks*block*block],
    off=dict(N, nnz, row_ptr, col, val))."""
    N = csr["N"]
    nblk = (N + block - 1) // block
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(csr["row_ptr"]))
    cols = csr["col"].astype(np.int64)
    inside = (rows // block) == (cols // block)
    diag = np.zeros(nblk * block * block, dtype=np.float64)
    ri, ci = rows[inside], cols[inside]
    # duplicate (row, column) entries add up, as they do in the CSR product
    np.add.at(diag, (ri // block) * block * block + (ri % block) * block + (ci % block), csr["val"][inside])
    out_rows = rows[~inside]
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(out_rows, minlength=N), out=row_ptr[1:])
    off = dict(N=N, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=csr["col"][~inside].copy(),
               val=csr["val"][~inside].copy())
    return dict(block=block, n_blocks=nblk, diag=diag, off=off)
