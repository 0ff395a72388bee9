"""The hand-written dense symmetric eigensolver (chfsi_eigh: Householder
tridiagonalisation, divide and conquer, blocked back-transformation) against
LAPACK (numpy.linalg.eigh) on random, clustered, degenerate and structured
symmetric matrices: eigenvalues to 1e-12 of the spectral radius, residuals
|A Q - Q diag(w)| / |A| and the orthogonality of Q to 1e-12."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2110_15853_gb300 import build
    build.build()
    import paper_2110_15853_gb300 as P
    return P


def _check(P, A, tol=1e-12):
    w, Q = P.eigh(torch.as_tensor(A).cuda())
    w, Q = w.cpu().numpy(), Q.cpu().numpy()
    ref = np.linalg.eigvalsh(A)
    scale = max(np.max(np.abs(ref)), 1e-300)
    n = A.shape[0]
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - ref)) <= tol * scale
    assert np.linalg.norm(A @ Q - Q * w) <= tol * max(np.linalg.norm(A), 1e-300) * max(1.0, np.sqrt(n) / 10)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= tol


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 64, 65, 100, 257, 1000])
def test_eigh_random(P, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    _check(P, (A + A.T) / 2)


def test_eigh_clustered_and_degenerate(P):
    rng = np.random.default_rng(7)
    n = 300
    Qr, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.linspace(-1.0, 2.0, n // 6), 6) + 1e-13 * rng.standard_normal(n)   # 6-fold clusters
    _check(P, (Qr * lam) @ Qr.T)
    lam = np.concatenate([np.zeros(100), np.ones(150), np.full(50, 3.0)])                 # exact degeneracy
    _check(P, (Qr * lam) @ Qr.T)


def test_eigh_structured(P):
    n = 200
    # Wilkinson-like tridiagonal (pairs of close eigenvalues), a diagonal matrix, a graded matrix
    W = np.diag(np.abs(np.arange(n) - n / 2)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    _check(P, W)
    _check(P, np.diag(np.linspace(5.0, -5.0, n)))
    rng = np.random.default_rng(3)
    G = rng.standard_normal((n, n))
    G = (G + G.T) / 2 * np.outer(np.logspace(0, -6, n), np.logspace(0, -6, n))
    _check(P, G)


def test_eigh_zero_matrix(P):
    w, Q = P.eigh(torch.zeros(40, 40, dtype=torch.float64, device="cuda"))
    assert torch.all(w == 0)
    assert np.max(np.abs(Q.cpu().numpy().T @ Q.cpu().numpy() - np.eye(40))) <= 1e-12


@pytest.mark.parametrize("n", [2048, 2100])
def test_eigh_blocked_tridiagonalisation(P, n):
    """n >= 2048 takes the blocked tridiagonalisation (panels of 32 reflectors, the
    trailing matrix updated once per panel): random symmetric matrices, a full panel
    count (2048) and a ragged last panel (2100)."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    _check(P, (A + A.T) / 2)


def test_eigh_blocked_clustered(P):
    rng = np.random.default_rng(11)
    n = 2200
    Qr, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.linspace(-3.0, 1.0, n // 8), 8) + 1e-12 * rng.standard_normal(n)
    _check(P, (Qr * lam) @ Qr.T)
