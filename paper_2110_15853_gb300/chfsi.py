"""Thin PyTorch binding of the chfsi C ABI (argument marshalling only).

Torch provides device memory and streams; every step of the filter, the
closure, the bounds and the adjoint runs in libchfsi.so kernels.  The binding
names follow the C entry points:

    filter(H, X, m, a, b, a0, schedule=None)            -> Y_m       (Algorithm 1, step 1)
    filter_backward(H, X, dY, m, a, b, a0, ...)         -> dX, dH     (reverse mode of step 1)
    rayleigh_ritz(H, Y, cholqr_passes=2)                -> ritz, Psi  (Algorithm 1, steps 2-5)
    lanczos_bounds(H, v0, steps, n_wanted)              -> a, b, a0   (bounds Algorithm 1 takes)
    ChebyshevFilter.apply(X, h_val, H, m, a, b, a0)     -> Y_m with autograd into X and h_val

a = eps_ub^w (upper bound of the wanted spectrum), b = eps_ub^uw (upper bound of
the unwanted spectrum), a0 = eps_0 (lower bound of the wanted spectrum).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import (CHFSI_BF16_F32ACC, CHFSI_BSR, CHFSI_CSR, CHFSI_F32, CHFSI_F32X2, CHFSI_F40_OZAKI, CHFSI_F64,
                   CHFSI_F64_OZAKI, ChfsiError, check, load)

PRECISIONS = {"f64": CHFSI_F64, "f32": CHFSI_F32, "bf16": CHFSI_BF16_F32ACC, "f32x2": CHFSI_F32X2,
              "ozaki": CHFSI_F64_OZAKI, "ozaki40": CHFSI_F40_OZAKI}


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream_handle(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclass
class CsrMatrix:
    """CSR operator resident on the device (row_ptr int64, col int32, val float64)."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    n_rows: int

    @classmethod
    def from_arrays(cls, row_ptr, col, val, device="cuda") -> "CsrMatrix":
        rp = torch.as_tensor(np.ascontiguousarray(row_ptr, dtype=np.int64)).to(device)
        cl = torch.as_tensor(np.ascontiguousarray(col, dtype=np.int32)).to(device)
        vl = torch.as_tensor(np.ascontiguousarray(val, dtype=np.float64)).to(device)
        return cls(rp, cl, vl, int(rp.shape[0] - 1))

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def device(self) -> torch.device:
        return self.val.device

    def descriptor(self, val: Optional[torch.Tensor] = None) -> _abi.chfsi_matrix:
        v = self.val if val is None else val
        m = _abi.chfsi_matrix()
        m.kind = CHFSI_CSR
        m.csr = _abi.chfsi_csr(self.n_rows, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(v))
        return m


@dataclass
class BsrMatrix:
    """Blocked CSR (64 x 64 dense blocks) resident on the device."""
    brow_ptr: torch.Tensor
    bcol: torch.Tensor
    val: torch.Tensor
    n_block_rows: int
    bdim: int = 64

    @classmethod
    def from_arrays(cls, brow_ptr, bcol, val, bdim=64, device="cuda") -> "BsrMatrix":
        bp = torch.as_tensor(np.ascontiguousarray(brow_ptr, dtype=np.int32)).to(device)
        bc = torch.as_tensor(np.ascontiguousarray(bcol, dtype=np.int32)).to(device)
        vl = torch.as_tensor(np.ascontiguousarray(val, dtype=np.float64)).to(device)
        return cls(bp, bc, vl, int(bp.shape[0] - 1), bdim)

    @property
    def n_rows(self) -> int:
        return self.n_block_rows * self.bdim

    @property
    def n_blocks(self) -> int:
        return int(self.bcol.shape[0])

    @property
    def device(self) -> torch.device:
        return self.val.device

    def descriptor(self, val: Optional[torch.Tensor] = None) -> _abi.chfsi_matrix:
        v = self.val if val is None else val
        m = _abi.chfsi_matrix()
        m.kind = CHFSI_BSR
        m.bsr = _abi.chfsi_bsr(self.n_block_rows, self.n_blocks, self.bdim, _ptr(self.brow_ptr), _ptr(self.bcol),
                               _ptr(v))
        return m


@dataclass
class HybridMatrix:
    """One operator in both layouts (CSR rows in the blocked order of the BSR):
    FP64/FP32 steps use the CSR, BF16-operand steps the BSR blocks on tensor cores."""
    csr: CsrMatrix
    bsr: BsrMatrix

    @property
    def n_rows(self) -> int:
        return self.csr.n_rows

    @property
    def nnz(self) -> int:
        return self.csr.nnz

    @property
    def device(self) -> torch.device:
        return self.csr.device

    def descriptor(self, val: Optional[torch.Tensor] = None) -> _abi.chfsi_matrix:
        m = _abi.chfsi_matrix()
        m.kind = _abi.CHFSI_HYBRID
        m.csr = self.csr.descriptor(val).csr
        m.bsr = self.bsr.descriptor().bsr
        return m


def _block_density(rows: np.ndarray, cols: np.ndarray, N: int, block: int) -> float:
    inside = int(np.count_nonzero(rows // block == cols // block))
    full, rem = divmod(N, block)
    return inside / float(full * block * block + rem * rem)


def split_block_density(row_ptr, col, block: int) -> float:
    """Fraction of the diagonal blocks' entries (blocks of `block` rows, the last one
    ragged) that the operator stores: the density the paper compares with 5% when it
    chooses the rows of a dense diagonal block H^{L(D)} (Sec. 4.1)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = len(row_ptr) - 1
    if N <= 0:
        return 0.0
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(row_ptr))
    return _block_density(rows, np.asarray(col, dtype=np.int64), N, int(block))


def split_block_size(row_ptr, col, min_density: float = 0.05, max_block: int = 8192) -> int:
    """The largest diagonal-block size among 128, 256, ..., max_block (and no larger
    than N rounded up to 128) whose diagonal blocks are at least `min_density` dense.
    Sec. 4.1 sizes the dense diagonal block as large as memory allows while its density
    stays above 5%, the point above which dense products beat sparse ones; 128 is the
    fallback when no size reaches the threshold."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = len(row_ptr) - 1
    if N <= 0:
        return 128
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(row_ptr))
    cols = np.asarray(col, dtype=np.int64)
    top = min(int(max_block), (N + 127) // 128 * 128)
    best, B = 128, 128
    while B <= top:
        if _block_density(rows, cols, N, B) >= min_density:
            best = B
        B *= 2
    return best


@dataclass
class SplitMatrix:
    """The paper's split storage (Sec. 4.1-4.2): dense block x block diagonal blocks
    (stacked, row-major) and the off-diagonal entries in CSR, resident on the device.
    Accepted by the filter (FP64 schedule); the dense blocks run on the tensor cores."""
    diag: torch.Tensor
    off: CsrMatrix
    block: int
    n_rows: int

    @classmethod
    def from_arrays(cls, diag, block, off_row_ptr, off_col, off_val, device="cuda") -> "SplitMatrix":
        off = CsrMatrix.from_arrays(off_row_ptr, off_col, off_val, device=device)
        dg = torch.as_tensor(np.ascontiguousarray(diag, dtype=np.float64)).to(device)
        return cls(dg, off, int(block), off.n_rows)

    @classmethod
    def from_csr(cls, row_ptr, col, val, block: Optional[int] = None, min_density: float = 0.05,
                 device="cuda") -> "SplitMatrix":
        """Split a host CSR operator: the entries whose column falls in the row's own
        block of `block` rows go to the dense diagonal blocks (duplicates add up), the rest
        stay in CSR.  Without `block`, the block is split_block_size(row_ptr, col,
        min_density)."""
        row_ptr = np.asarray(row_ptr, dtype=np.int64)
        col = np.asarray(col)
        val = np.asarray(val, dtype=np.float64)
        N = len(row_ptr) - 1
        B = int(block) if block is not None else split_block_size(row_ptr, col, min_density)
        nblk = (N + B - 1) // B
        rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(row_ptr))
        cols = col.astype(np.int64)
        inside = (rows // B) == (cols // B)
        diag = np.zeros(nblk * B * B, dtype=np.float64)
        ri, ci = rows[inside], cols[inside]
        np.add.at(diag, (ri // B) * B * B + (ri % B) * B + (ci % B), val[inside])
        off_ptr = np.zeros(N + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows[~inside], minlength=N), out=off_ptr[1:])
        return cls.from_arrays(diag, B, off_ptr, col[~inside].astype(np.int32), val[~inside], device=device)

    @property
    def device(self) -> torch.device:
        return self.diag.device

    def descriptor(self, val: Optional[torch.Tensor] = None) -> _abi.chfsi_matrix:
        m = _abi.chfsi_matrix()
        m.kind = _abi.CHFSI_SPLIT
        m.split = _abi.chfsi_split(self.n_rows, self.block, _ptr(self.diag), self.off.descriptor().csr)
        return m


class Workspace:
    """Grow-only device scratch buffer (allocate once, outside timed loops)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf: Optional[torch.Tensor] = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


def _schedule(m: int, schedule: Optional[Sequence]) -> Optional[ctypes.Structure]:
    if schedule is None:
        return None
    codes = [PRECISIONS[p] if isinstance(p, str) else int(p) for p in schedule]
    if len(codes) != m:
        raise ValueError("schedule must list one precision per step")
    arr = (ctypes.c_int32 * m)(*codes)
    s = _abi.chfsi_schedule(m, ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)))
    s._keep = arr
    return s


def mixed_schedule(m: int, low_steps: int, low: str = "f32") -> list:
    """low_steps leading steps in `low` precision, the rest FP64."""
    return [low] * low_steps + ["f64"] * (m - low_steps)


def _check_block(t: torch.Tensor, name: str) -> None:
    if t.dtype != torch.float64 or t.dim() != 2 or t.stride(1) != 1 or not t.is_cuda:
        raise ValueError(f"{name} must be a row-major (N, n) float64 CUDA tensor")


def filter_workspace_bytes(H, n_cols: int, m: int, schedule=None) -> int:
    sz = ctypes.c_size_t(0)
    desc = H.descriptor()
    check(load().chfsi_filter_workspace_size(ctypes.byref(desc), n_cols, m, _schedule(m, schedule),
                                             ctypes.byref(sz)), "chfsi_filter_workspace_size")
    return sz.value


def filter(H, X: torch.Tensor, m: int, a: float, b: float, a0: float, schedule=None,
           out: Optional[torch.Tensor] = None, workspace: Optional[Workspace] = None) -> torch.Tensor:
    """Y_m of the scaled Chebyshev filter (Algorithm 1 step 1) on the GPU.

    schedule: None (every step FP64) or one precision per step, by name or code:
    "f64"; "f32", "bf16", "f32x2" (a leading low-precision prefix of one kind); "ozaki"
    (FP64-accurate products on the tensor cores) and "ozaki40" (40-bit Ozaki products),
    in any order after the prefix, for operators with 64 x 64 blocks (BsrMatrix or
    HybridMatrix).  The rules are chfsi_filter's (include/chfsi.h)."""
    _check_block(X, "X")
    N, n = X.shape
    if out is None:
        out = torch.empty((N, n), dtype=torch.float64, device=X.device)
    _check_block(out, "out")
    lib = load()
    desc = H.descriptor()
    sch = _schedule(m, schedule)
    ws = (workspace or Workspace(X.device)).get(filter_workspace_bytes(H, n, m, schedule))
    rc = lib.chfsi_filter(ctypes.byref(desc), _ptr(X), X.stride(0), _ptr(out), out.stride(0), n, m, a, b, a0,
                          sch, _ptr(ws), ws.numel(), _stream_handle(X.device))
    check(rc, "chfsi_filter")
    return out


def read_status(workspace: Workspace) -> int:
    return load().chfsi_read_status(_ptr(workspace.buf), _stream_handle(workspace.device))


def filter_backward(H: CsrMatrix, X: torch.Tensor, dY: torch.Tensor, m: int, a: float, b: float, a0: float,
                    ckpt_stride: int = 0, want_dH: bool = True, val: Optional[torch.Tensor] = None,
                    workspace: Optional[Workspace] = None, precision: str = "f64"):
    """(dX, dH_val) for dL/dY_m = dY; dH_val has one entry per stored entry of H.

    precision "f64" (chfsi_filter_backward) or "f32x2" (two-float sweep,
    chfsi_filter_backward_ex)."""
    _check_block(X, "X")
    _check_block(dY, "dY")
    N, n = X.shape
    lib = load()
    desc = H.descriptor(val)
    sz = ctypes.c_size_t(0)
    code = PRECISIONS[precision]
    check(lib.chfsi_filter_backward_ex_workspace_size(ctypes.byref(desc), n, m, ckpt_stride, code,
                                                      ctypes.byref(sz)), "chfsi_filter_backward_ex_workspace_size")
    ws = (workspace or Workspace(X.device)).get(sz.value)
    dX = torch.empty((N, n), dtype=torch.float64, device=X.device)
    dH = torch.empty(H.nnz, dtype=torch.float64, device=X.device) if want_dH else None
    args = (ctypes.byref(desc), _ptr(X), X.stride(0), _ptr(dY), dY.stride(0), _ptr(dX), dX.stride(0), _ptr(dH), n, m,
            a, b, a0, ckpt_stride)
    if precision == "f64":
        rc = lib.chfsi_filter_backward(*args, _ptr(ws), ws.numel(), _stream_handle(X.device))
        check(rc, "chfsi_filter_backward")
    else:
        rc = lib.chfsi_filter_backward_ex(*args, code, _ptr(ws), ws.numel(), _stream_handle(X.device))
        check(rc, "chfsi_filter_backward_ex")
    return dX, dH


def rayleigh_ritz_workspace_bytes(H, n_cols: int, cholqr_passes: int = 2, precision: str = "f64") -> int:
    sz = ctypes.c_size_t(0)
    desc = H.descriptor()
    check(load().chfsi_rayleigh_ritz_ex_workspace_size(ctypes.byref(desc), n_cols, cholqr_passes,
                                                       PRECISIONS[precision], ctypes.byref(sz)),
          "chfsi_rayleigh_ritz_ex_workspace_size")
    return sz.value


def rayleigh_ritz(H, Y: torch.Tensor, cholqr_passes: int = 2, psi: Optional[torch.Tensor] = None,
                  ritz: Optional[torch.Tensor] = None, workspace: Optional[Workspace] = None,
                  precision: str = "f64"):
    """(ritz ascending, Psi) from Algorithm 1 steps 2-5 (CholQR, projection, eig, rotation).

    precision "f64" runs every product in FP64 (chfsi_rayleigh_ritz); "f32x2" runs
    the large products in two-float arithmetic and "ozaki" the dense products on the
    BF16 tensor cores by Ozaki slices (chfsi_rayleigh_ritz_ex)."""
    _check_block(Y, "Y")
    N, n = Y.shape
    if psi is None:
        psi = torch.empty((N, n), dtype=torch.float64, device=Y.device)
    if ritz is None:
        ritz = torch.empty(n, dtype=torch.float64, device=Y.device)
    lib = load()
    desc = H.descriptor()
    ws = (workspace or Workspace(Y.device)).get(rayleigh_ritz_workspace_bytes(H, n, cholqr_passes, precision))
    args = (ctypes.byref(desc), _ptr(Y), Y.stride(0), n, _ptr(psi), psi.stride(0), _ptr(ritz), cholqr_passes)
    if precision == "f64":
        rc = lib.chfsi_rayleigh_ritz(*args, _ptr(ws), ws.numel(), _stream_handle(Y.device))
        check(rc, "chfsi_rayleigh_ritz")
    else:
        rc = lib.chfsi_rayleigh_ritz_ex(*args, PRECISIONS[precision], _ptr(ws), ws.numel(),
                                        _stream_handle(Y.device))
        check(rc, "chfsi_rayleigh_ritz_ex")
    return ritz, psi


def ozaki_gemm(A: torch.Tensor, B: torch.Tensor, transpose_a: bool = False, symmetric: bool = False,
               b_upper: bool = False, out: Optional[torch.Tensor] = None,
               workspace: Optional[Workspace] = None) -> torch.Tensor:
    """FP64-accurate product on the BF16 tensor cores (chfsi_ozaki_gemm):
    A^T B if transpose_a (A: K x M, B: K x Nc) else A B (A: M x K, B: K x Nc)."""
    for t, name in ((A, "A"), (B, "B")):
        if t.dtype != torch.float64 or t.dim() != 2 or t.stride(1) != 1 or not t.is_cuda:
            raise ValueError(f"{name} must be a row-major float64 CUDA matrix")
    if transpose_a:
        K, M = A.shape
    else:
        M, K = A.shape
    if B.shape[0] != K:
        raise ValueError("inner dimensions differ")
    Nc = B.shape[1]
    op = _abi.CHFSI_OP_TN if transpose_a else _abi.CHFSI_OP_NN
    flags = (_abi.CHFSI_GEMM_SYMMETRIC if symmetric else 0) | (_abi.CHFSI_GEMM_B_UPPER if b_upper else 0)
    if out is None:
        out = torch.empty((M, Nc), dtype=torch.float64, device=A.device)
    lib = load()
    sz = ctypes.c_size_t(0)
    check(lib.chfsi_ozaki_gemm_workspace_size(op, M, Nc, K, flags, ctypes.byref(sz)),
          "chfsi_ozaki_gemm_workspace_size")
    ws = (workspace or Workspace(A.device)).get(sz.value)
    check(lib.chfsi_ozaki_gemm(op, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(out), out.stride(0), M, Nc, K,
                               flags, _ptr(ws), ws.numel(), _stream_handle(A.device)), "chfsi_ozaki_gemm")
    return out


def eigh(A: torch.Tensor, workspace: Optional[Workspace] = None):
    """(w ascending, Q) of a symmetric FP64 CUDA matrix by the library's dense
    eigensolver (chfsi_eigh); A is not modified (a copy is factorised)."""
    if A.dtype != torch.float64 or A.dim() != 2 or A.shape[0] != A.shape[1] or not A.is_cuda:
        raise ValueError("A must be a square float64 CUDA matrix")
    n = A.shape[0]
    work = A.contiguous().clone()
    w = torch.empty(n, dtype=torch.float64, device=A.device)
    Q = torch.empty((n, n), dtype=torch.float64, device=A.device)
    lib = load()
    sz = ctypes.c_size_t(0)
    check(lib.chfsi_eigh_workspace_size(n, ctypes.byref(sz)), "chfsi_eigh_workspace_size")
    ws = (workspace or Workspace(A.device)).get(sz.value)
    check(lib.chfsi_eigh(_ptr(work), n, n, _ptr(w), _ptr(Q), n, _ptr(ws), ws.numel(), _stream_handle(A.device)),
          "chfsi_eigh")
    return w, Q


def measure_pipe_peak(precision: str = "f64", device="cuda") -> float:
    """FLOP/s of the FP64 (DFMA) or FP32 (FFMA) pipe of `device`, measured by the
    library's register-resident FMA loop (chfsi_measure_pipe_peak)."""
    out = ctypes.c_double(0.0)
    dev = torch.device(device)
    with torch.cuda.device(dev):
        check(load().chfsi_measure_pipe_peak(PRECISIONS[precision], ctypes.byref(out), _stream_handle(dev)),
              "chfsi_measure_pipe_peak")
    return out.value


def lanczos_workspace_bytes(H, steps: int) -> int:
    sz = ctypes.c_size_t(0)
    desc = H.descriptor()
    check(load().chfsi_lanczos_workspace_size(ctypes.byref(desc), steps, ctypes.byref(sz)),
          "chfsi_lanczos_workspace_size")
    return sz.value


def lanczos_bounds(H: CsrMatrix, v0: torch.Tensor, steps: int, n_wanted: int,
                   workspace: Optional[Workspace] = None):
    """(a, b, a0) from `steps` Lanczos steps started at v0 (device float64, length N)."""
    if v0.dtype != torch.float64 or not v0.is_cuda or v0.dim() != 1:
        raise ValueError("v0 must be a 1-D float64 CUDA tensor")
    lib = load()
    desc = H.descriptor()
    sz = ctypes.c_size_t(0)
    check(lib.chfsi_lanczos_workspace_size(ctypes.byref(desc), steps, ctypes.byref(sz)),
          "chfsi_lanczos_workspace_size")
    ws = (workspace or Workspace(v0.device)).get(sz.value)
    a, b, a0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.chfsi_lanczos_bounds(ctypes.byref(desc), steps, _ptr(v0.contiguous()), n_wanted, ctypes.byref(a),
                                  ctypes.byref(b), ctypes.byref(a0), _ptr(ws), ws.numel(), _stream_handle(v0.device))
    check(rc, "chfsi_lanczos_bounds")
    return a.value, b.value, a0.value


def solve(H, X: torch.Tensor, m: int, cycles: int, v0: torch.Tensor, lanczos_steps: int = 20, schedule=None,
          rr_precision: str = "f64", cholqr_passes: int = 2, workspace: Optional[Workspace] = None):
    """Repeated ChFSI cycles: Algorithm 1 applied again with the previous cycle's
    Psi as X (Sec. 3.4: later SCF iterations start from the previous Psi).

    Cycle 1 takes its bounds from chfsi_lanczos_bounds; later cycles use the
    Zhou-Saad update a0 = smallest and a = largest Ritz value of the previous
    cycle, with b (the Lanczos upper bound of the spectrum) kept.  Returns
    (ritz, Psi, history) with history[i] the Ritz values after cycle i + 1.
    """
    N, n = X.shape
    ws_f, ws_r = workspace or Workspace(X.device), Workspace(X.device)
    a, b, a0 = lanczos_bounds(H, v0, lanczos_steps, n, workspace=ws_f)
    Y = torch.empty_like(X)
    psi = X.clone()
    ritz = torch.empty(n, dtype=torch.float64, device=X.device)
    history = []
    for _ in range(cycles):
        filter(H, psi, m, a, b, a0, schedule=schedule, out=Y, workspace=ws_f)
        ritz, psi = rayleigh_ritz(H, Y, cholqr_passes, psi=psi, ritz=ritz, workspace=ws_r, precision=rr_precision)
        history.append(ritz.clone())
        a0, a = float(ritz[0]), float(ritz[-1])
    return ritz, psi, history


class ChebyshevFilter(torch.autograd.Function):
    """Y_m = p(H) X with gradients into X and into H's stored values.

    The bounds a, b, a0 are constants (no gradient).  The backward pass is the
    hand-written adjoint (chfsi_filter_backward) with sqrt(m) checkpointing; it
    uses H for H^T, so H must be symmetric.
    """

    @staticmethod
    def forward(ctx, X, h_val, H: CsrMatrix, m: int, a: float, b: float, a0: float, ckpt_stride: int = 0):
        ctx.H, ctx.m, ctx.a, ctx.b, ctx.a0, ctx.ckpt = H, m, a, b, a0, ckpt_stride
        Xc = X.detach().contiguous()
        hv = h_val.detach().contiguous()
        ctx.save_for_backward(Xc, hv)
        H_eff = CsrMatrix(H.row_ptr, H.col, hv, H.n_rows)
        return filter(H_eff, Xc, m, a, b, a0)

    @staticmethod
    def backward(ctx, gY):
        Xc, hv = ctx.saved_tensors
        H_eff = CsrMatrix(ctx.H.row_ptr, ctx.H.col, hv, ctx.H.n_rows)
        dX, dH = filter_backward(H_eff, Xc, gY.contiguous(), ctx.m, ctx.a, ctx.b, ctx.a0, ctx.ckpt,
                                 want_dH=ctx.needs_input_grad[1])
        return (dX if ctx.needs_input_grad[0] else None, dH, None, None, None, None, None, None)


def symmetric_gradient(H: CsrMatrix, dH: torch.Tensor, transpose_index: torch.Tensor) -> torch.Tensor:
    """dH_sym[p] = dH[p] + dH[p^T] off the diagonal, dH[p] on it, for a symmetric
    parameterisation where entries (i, j) and (j, i) share one value."""
    out = dH + dH[transpose_index]
    diag = transpose_index == torch.arange(dH.shape[0], device=dH.device)
    return torch.where(diag, dH, out)


def transpose_index(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """For a structurally symmetric CSR pattern: index of entry (j, i) for each (i, j).

    Raises ValueError if an entry (i, j) has no stored (j, i), or if a pattern
    stores the same (i, j) twice (the pairing would then not be one to one)."""
    N = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(N, dtype=np.int64), np.diff(row_ptr))
    key = rows * N + col.astype(np.int64)
    tkey = col.astype(np.int64) * N + rows
    order = np.argsort(key, kind="stable")
    skey = key[order]
    if skey.size > 1 and np.any(skey[1:] == skey[:-1]):
        raise ValueError("transpose_index: the pattern stores an entry (i, j) more than once")
    pos = np.searchsorted(skey, tkey)
    found = pos < skey.size
    found[found] = skey[pos[found]] == tkey[found]
    if not np.all(found):
        raise ValueError("transpose_index: the pattern is not structurally symmetric")
    return order[pos]
