"""FP64 CPU oracle for the ChFSI filter path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product library (``paper_2110_15853_gb300``) never
imports it and shares no code with it.

What it computes (all FP64):

* ``spmm`` / ``spmm_t`` -- H X and H^T X for CSR H, row by row in stored order
  (plain C, ``chfsi_oracle.c``, compiled with -ffp-contract=off).
* ``filter`` -- the scaled Chebyshev filter of Algorithm 1 step 1 (Sec. 3.4), as the
  three-term recurrence Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2}.
* ``filter_adjoint`` -- reverse-mode derivative of that loop, all iterates stored.
* ``lanczos_bounds`` -- k-step Lanczos with full re-orthogonalisation giving the
  bounds (eps_0, eps_ub^w, eps_ub^uw) = (a0, a, b) that Algorithm 1 takes as input
  (the paper does not say how they are obtained; the reading used is documented
  in the function).
* ``rayleigh_ritz`` -- Algorithm 1 steps 2-5 with Householder QR (LAPACK) as the
  orthonormalisation, the projection X_F^T H X_F, a LAPACK symmetric eigensolve
  and the rotation Psi = X_F Q.

Pinned by tests/test_oracle_pins.py against closed forms (diagonal H, H = Q
diag(lambda) Q^T, Kronecker sums), invariants, brute-force eigensolves,
complex-step derivatives and the Daleckii-Krein formula.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chfsi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile chfsi_oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_spmm.argtypes = [i64, _i64p, _i32p, _dp, i64, _dp, i64, _dp, i64]
        lib.oracle_spmm_t.argtypes = [i64, _i64p, _i32p, _dp, i64, _dp, i64, _dp, i64]
        lib.oracle_filter.argtypes = [i64, _i64p, _i32p, _dp, i64, _dp, i64, i32, dbl, dbl, dbl,
                                      _dp, i64, _dp]
        lib.oracle_filter.restype = ctypes.c_int
        lib.oracle_filter_adjoint.argtypes = [i64, _i64p, _i32p, _dp, i64, _dp, i64, i32, dbl, dbl,
                                              dbl, _dp, i64, _dp, i64, _dp, _dp]
        lib.oracle_filter_adjoint.restype = ctypes.c_int
        lib.oracle_coefficients.argtypes = [i32, dbl, dbl, dbl, _dp, _dp, _dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr(H):
    rp = np.ascontiguousarray(H["row_ptr"], dtype=np.int64)
    col = np.ascontiguousarray(H["col"], dtype=np.int32)
    val = np.ascontiguousarray(H["val"], dtype=np.float64)
    return int(rp.shape[0] - 1), rp, col, val


def _block(X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    return X


def spmm(H, X) -> np.ndarray:
    """H X (CSR H, row by row in stored column order)."""
    N, rp, col, val = _csr(H)
    squeeze = np.ndim(X) == 1
    X = _block(X)
    n = X.shape[1]
    Y = np.empty((N, n))
    _load().oracle_spmm(N, _p(rp, _i64p), _p(col, _i32p), _p(val, _dp), n, _p(X, _dp), n,
                        _p(Y, _dp), n)
    return Y[:, 0] if squeeze else Y


def spmm_t(H, X) -> np.ndarray:
    """H^T X (scatter of every stored entry into its column's row)."""
    N, rp, col, val = _csr(H)
    X = _block(X)
    n = X.shape[1]
    Y = np.empty((N, n))
    _load().oracle_spmm_t(N, _p(rp, _i64p), _p(col, _i32p), _p(val, _dp), n, _p(X, _dp), n,
                          _p(Y, _dp), n)
    return Y


def coefficients(m: int, a: float, b: float, a0: float):
    """(alpha[0..m], beta[0..m], c) of Y_k = alpha_k (H - c) Y_{k-1} - beta_k Y_{k-2}."""
    alpha = np.zeros(m + 1)
    beta = np.zeros(m + 1)
    c = ctypes.c_double(0.0)
    _load().oracle_coefficients(int(m), float(a), float(b), float(a0), _p(alpha, _dp),
                                _p(beta, _dp), ctypes.byref(c))
    return alpha, beta, c.value


def filter(H, X, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Y_m of Algorithm 1 step 1 (a = eps_ub^w, b = eps_ub^uw, a0 = eps_0)."""
    N, rp, col, val = _csr(H)
    X = _block(X)
    n = X.shape[1]
    Y = np.empty((N, n))
    work = np.empty(3 * N * n)
    rc = _load().oracle_filter(N, _p(rp, _i64p), _p(col, _i32p), _p(val, _dp), n, _p(X, _dp), n,
                               int(m), float(a), float(b), float(a0), _p(Y, _dp), n,
                               _p(work, _dp))
    if rc != 0:
        raise ValueError("oracle filter: degree m must be >= 1")
    return Y


def filter_adjoint(H, X, m: int, a: float, b: float, a0: float, G, want_dH: bool = True):
    """(dX, dH) for dL/dY_m = G; dH holds one value per stored entry of H."""
    N, rp, col, val = _csr(H)
    X = _block(X)
    G = _block(G)
    n = X.shape[1]
    dX = np.empty((N, n))
    dH = np.empty(val.shape[0]) if want_dH else None
    work = np.empty((m + 4) * N * n)
    rc = _load().oracle_filter_adjoint(
        N, _p(rp, _i64p), _p(col, _i32p), _p(val, _dp), n, _p(X, _dp), n, int(m), float(a),
        float(b), float(a0), _p(G, _dp), n, _p(dX, _dp), n,
        _p(dH, _dp) if want_dH else ctypes.cast(None, _dp), _p(work, _dp))
    if rc != 0:
        raise ValueError("oracle adjoint: degree m must be >= 1")
    return dX, dH


def lanczos(H, v0, steps: int, return_basis: bool = False):
    """k-step Lanczos with full re-orthogonalisation.

    v_1 = v0/|v0|; for j = 1..k: w = H v_j, alpha_j = v_j^T w,
    w -= alpha_j v_j + beta_{j-1} v_{j-1}, then w -= V_j (V_j^T w) (one classical
    Gram-Schmidt pass against all previous vectors), beta_j = |w|, v_{j+1} = w/beta_j.
    k = min(steps, N).  Breakdown (beta_j <= 1e-12 times the largest
    |alpha_i| + beta_{i-1} seen so far) ends the iteration with a zero residual.
    Returns (alpha[k], beta[k]) where beta[k-1] is the final residual norm, plus
    the basis V (k x N) when return_basis is set.
    """
    N = int(H["row_ptr"].shape[0] - 1)
    k = min(int(steps), N)
    V = np.zeros((k + 1, N))
    al = np.zeros(k)
    be = np.zeros(k)
    V[0] = v0 / np.linalg.norm(v0)
    scale = 0.0
    for j in range(k):
        w = spmm(H, V[j])
        al[j] = V[j] @ w
        w = w - al[j] * V[j]
        if j > 0:
            w = w - be[j - 1] * V[j - 1]
        w = w - V[: j + 1].T @ (V[: j + 1] @ w)
        be[j] = np.linalg.norm(w)
        scale = max(scale, abs(al[j]) + (be[j - 1] if j > 0 else 0.0))
        if be[j] <= 1e-12 * scale:
            be[j] = 0.0
            k = j + 1
            break
        V[j + 1] = w / be[j]
    if return_basis:
        return al[:k], be[:k], V[:k]
    return al[:k], be[:k]


def lanczos_bounds(H, v0, steps: int, n_wanted: int):
    """Bounds (a, b, a0) = (eps_ub^w, eps_ub^uw, eps_0) for Algorithm 1.

    theta = eig(T_k) ascending; a0 = theta_1; b = theta_k + |beta_k| (largest Ritz
    value plus the residual norm, Zhou-Saad's upper-bound safeguard);
    a = a0 + (b - a0) (n_wanted/N)^(2/3) (3-D Weyl law: the count of eigenvalues
    below lambda grows like (lambda - lambda_min)^(3/2)).
    """
    N = int(H["row_ptr"].shape[0] - 1)
    al, be = lanczos(H, v0, steps)
    theta = scipy.linalg.eigh_tridiagonal(al, be[:-1], eigvals_only=True)
    a0 = float(theta[0])
    b = float(theta[-1] + abs(be[-1]))
    a = a0 + (b - a0) * (float(n_wanted) / float(N)) ** (2.0 / 3.0)
    return a, b, a0


def rayleigh_ritz(H, Y):
    """Algorithm 1 steps 2-5: X_F = Orth(Y) (Householder QR), H_F = X_F^T H X_F,
    H_F Q = Q Lambda (ascending), Psi = X_F Q.  Returns (theta, Psi, X_F)."""
    Y = _block(Y)
    XF, _ = np.linalg.qr(Y)
    HXF = spmm(H, XF)
    HF = XF.T @ HXF
    theta, Q = scipy.linalg.eigh(HF, driver="evd")
    Psi = XF @ Q
    return theta, Psi, XF
