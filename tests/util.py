"""Small helpers for the tests (no filter arithmetic lives here)."""
import numpy as np


def dense_to_csr(A, keep_zeros=True):
    """Store every entry of a dense square matrix (or its nonzeros) in CSR."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    mask = np.ones_like(A, dtype=bool) if keep_zeros else (A != 0)
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    cols = np.nonzero(mask)[1].astype(np.int32)
    return dict(N=N, nnz=int(row_ptr[-1]), row_ptr=row_ptr, col=cols, val=A[mask].copy())


def csr_to_dense(H):
    N = H["N"] if "N" in H else H["row_ptr"].shape[0] - 1
    A = np.zeros((N, N))
    rows = np.repeat(np.arange(N), np.diff(H["row_ptr"]))
    A[rows, H["col"]] = H["val"]
    return A


def cheb_T(m, x):
    """Chebyshev T_m(x) from its trigonometric / hyperbolic closed form."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1.0
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.cosh(m * np.arccosh(np.abs(xo))) * np.sign(xo) ** m
    return out


def cheb_dT(m, x):
    """T_m'(x) = m U_{m-1}(x) from sin/sinh closed forms (x away from +-1)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) < 1.0
    th = np.arccos(x[inside])
    out[inside] = m * np.sin(m * th) / np.sin(th)
    xo = x[~inside]
    u = np.arccosh(np.abs(xo))
    out[~inside] = m * np.sinh(m * u) / np.sinh(u) * np.sign(xo) ** (m - 1)
    return out


def rel_fro(A, B):
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


def random_orthogonal(N, seed):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((N, N)))
    return Q * np.sign(np.diag(R))
