"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks retypes the oracle's own loop: each compares it with a
closed form (Chebyshev polynomials of a diagonal or spectrally known H, a
Kronecker-sum eigenbasis), an invariant (symmetry, linearity, column
independence, interlacing), a brute-force eigensolve, a complex-step or
finite-difference derivative, or the Daleckii-Krein formula.

The filter of Algorithm 1 (Sec. 3.4) applies p(H) = T_m((H - c)/e) / T_m(tau)
with tau = (a0 - c)/e: the sigma recurrence sigma_{k+1} = 1/(gamma - sigma_k),
gamma = 2/sigma_1 = 2 tau is the ratio T_k(tau)/T_{k+1}(tau), so each iterate is
Y_k = T_k(t(H))/T_k(tau) X.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import chfsi_workloads as W
from tests.util import cheb_T, cheb_dT, csr_to_dense, dense_to_csr, random_orthogonal, rel_fro


def p_of(lam, m, a, b, a0):
    e, c = (b - a) / 2.0, (b + a) / 2.0
    return cheb_T(m, (np.asarray(lam) - c) / e) / cheb_T(m, np.array([(a0 - c) / e]))[0]


def dp_of(lam, m, a, b, a0):
    e, c = (b - a) / 2.0, (b + a) / 2.0
    return cheb_dT(m, (np.asarray(lam) - c) / e) / e / cheb_T(m, np.array([(a0 - c) / e]))[0]


# --------------------------------------------------------------------------- filter


@pytest.mark.parametrize("m", [1, 2, 3, 7, 10, 20])
def test_diagonal_H_is_chebyshev_of_scaled_eigenvalues(oracle_mod, m):
    """On diagonal H each row is scaled by T_m((h_ii - c)/e)/T_m(tau)."""
    rng = np.random.default_rng(11)
    a0, a, b = 0.5, 1.7, 6.0
    d = np.concatenate([np.linspace(a0, a, 9), np.linspace(a, b, 17), [b + 0.3, a0 - 0.05]])
    N = d.size
    H = dense_to_csr(np.diag(d), keep_zeros=False)
    X = rng.standard_normal((N, 5))
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    pv = p_of(d, m, a, b, a0)[:, None]
    expect = pv * X
    # rounding of t = (d - c)/e moves T_m by at most ~m^2 ulp near the zeros of T_m
    tol = 5e-13 * np.abs(expect) + 1e-15 * m * m * np.abs(X) * np.maximum(1.0, np.abs(pv))
    assert np.all(np.abs(Y - expect) <= tol)


def test_chebyshev_inside_interval_is_cos_m_theta(oracle_mod):
    """T_m(cos theta) = cos(m theta): eigenvalues at Chebyshev nodes of [a, b]."""
    m, a0, a, b = 12, -3.0, -1.0, 5.0
    e, c = (b - a) / 2.0, (b + a) / 2.0
    theta = np.linspace(0.05, 3.0, 23)
    lam = c + e * np.cos(theta)
    H = dense_to_csr(np.diag(lam), keep_zeros=False)
    X = np.ones((lam.size, 1))
    Y = oracle_mod.filter(H, X, m, a, b, a0)[:, 0]
    tau = (a0 - c) / e
    Tm_tau = math.cosh(m * math.acosh(-tau)) * (-1) ** m
    assert np.max(np.abs(Y * Tm_tau - np.cos(m * theta))) < 1e-11


def test_textbook_T10_coefficients(oracle_mod):
    """1x1 H = [lambda]: the filter equals the integer-coefficient T_10 (tests/golden)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "chebyshev_T10.txt")
    coef = np.loadtxt(path, comments="#")          # highest power first
    a0, a, b = -2.0, -1.0, 1.0                      # e = 1, c = 0, t = lambda
    for lam in [-0.93, -0.4, 0.0, 0.21, 0.77, 1.0, 1.3, -1.6]:
        H = dense_to_csr(np.array([[lam]]))
        y = oracle_mod.filter(H, np.ones((1, 1)), 10, a, b, a0)[0, 0]
        expect = np.polyval(coef, lam) / np.polyval(coef, a0)
        assert abs(y - expect) <= 1e-12 * max(1.0, abs(expect))


@pytest.mark.parametrize("m", [1, 4, 10, 16])
def test_spectral_H_closed_form(oracle_mod, m):
    """H = Q diag(lambda) Q^T with known Q: Y_m = Q diag(p(lambda)) Q^T X."""
    N = 40
    Q = random_orthogonal(N, 5)
    lam = np.sort(np.random.default_rng(6).uniform(0.0, 10.0, N))
    a0, a, b = lam[0], lam[7], lam[-1] + 0.1
    A = Q @ np.diag(lam) @ Q.T
    A = 0.5 * (A + A.T)
    H = dense_to_csr(A)
    X = np.random.default_rng(7).standard_normal((N, 6))
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    expect = Q @ (p_of(lam, m, a, b, a0)[:, None] * (Q.T @ X))
    assert rel_fro(Y, expect) < 1e-12


def _kronecker_apply(g, w, fvals_fn, X):
    """Apply f(H0) for H0 = A(x)I(x)I + I(x)A(x)I + I(x)I(x)A via the 1-D eigenbasis."""
    A = np.zeros((g, g))
    for i in range(g):
        for j in range(g):
            d = abs(i - j)
            if d == 0:
                A[i, j] = 2.5
            elif d <= w:
                A[i, j] = -1.0 / (1.0 + d) ** 2
    mu, U = np.linalg.eigh(A)
    lam = mu[:, None, None] + mu[None, :, None] + mu[None, None, :]
    n = X.shape[1]
    T = X.reshape(g, g, g, n)
    T = np.einsum("ai,bj,ck,abcn->ijkn", U, U, U, T)
    T = T * fvals_fn(lam)[..., None]
    T = np.einsum("ai,bj,ck,ijkn->abcn", U, U, U, T)
    return T.reshape(g ** 3, n), lam


def test_kronecker_sum_closed_form_full_size(oracle_mod):
    """Potential-free 20^3, w=2 operator: exact eigenbasis u_i (x) u_j (x) u_k."""
    g, w, m = 20, 2, 10
    H = W.csr_grid(g, w, 0.0, 123)
    X = np.random.default_rng(8).standard_normal((g ** 3, 8))
    _, lam = _kronecker_apply(g, w, lambda l: l, X[:, :1])
    lmin, lmax = lam.min(), lam.max()
    a0, b = lmin, lmax + 1e-3
    a = a0 + (b - a0) * 0.1
    expect, _ = _kronecker_apply(g, w, lambda l: p_of(l, m, a, b, a0), X)
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    assert rel_fro(Y, expect) < 1e-12


def _small_case(g=8, w=2, n=6, seed=3):
    H = W.csr_grid(g, w, 0.1, seed)
    A = csr_to_dense(H)
    lam = np.linalg.eigvalsh(A)
    a0, b = lam[0], lam[-1]
    a = lam[g ** 3 // 8]
    X = np.random.default_rng(seed).standard_normal((g ** 3, n))
    return H, A, X, (a, b, a0)


def test_filter_matches_dense_eigendecomposition(oracle_mod):
    H, A, X, (a, b, a0) = _small_case()
    lam, Q = np.linalg.eigh(A)
    for m in (5, 13):
        Y = oracle_mod.filter(H, X, m, a, b, a0)
        expect = Q @ (p_of(lam, m, a, b, a0)[:, None] * (Q.T @ X))
        assert rel_fro(Y, expect) < 1e-12


def test_filter_symmetry_linearity_columns(oracle_mod):
    H, _, X, (a, b, a0) = _small_case(g=12, w=3, n=7, seed=4)
    m = 9
    Z = np.random.default_rng(9).standard_normal(X.shape)
    pX = oracle_mod.filter(H, X, m, a, b, a0)
    pZ = oracle_mod.filter(H, Z, m, a, b, a0)
    # symmetry of p(H):  Z^T p(H) X = (p(H) Z)^T X
    assert rel_fro(Z.T @ pX, pZ.T @ X) < 1e-12
    # linearity
    pc = oracle_mod.filter(H, 2.5 * X - 0.75 * Z, m, a, b, a0)
    assert rel_fro(pc, 2.5 * pX - 0.75 * pZ) < 1e-12
    # column independence: a column subset filters to the same columns, bit for bit
    cols = [0, 3, 6]
    assert np.array_equal(oracle_mod.filter(H, X[:, cols], m, a, b, a0), pX[:, cols])
    # m = 1 is one scaled, shifted product
    Y1 = oracle_mod.filter(H, X, 1, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2
    A = csr_to_dense(H)
    assert rel_fro(Y1, (e / (a0 - c)) / e * (A @ X - c * X)) < 1e-13


def test_filter_rejects_degree_zero(oracle_mod):
    H, _, X, (a, b, a0) = _small_case(g=4, w=1, n=2)
    with pytest.raises(ValueError):
        oracle_mod.filter(H, X, 0, a, b, a0)


def test_spmm_and_transpose_against_dense(oracle_mod):
    H, A, X, _ = _small_case(g=6, w=2, n=5)
    assert rel_fro(oracle_mod.spmm(H, X), A @ X) < 1e-14
    # a non-symmetric pattern-preserving perturbation distinguishes H and H^T
    Hn = dict(H)
    Hn["val"] = H["val"] * (1.0 + 0.1 * np.arange(H["nnz"]) / H["nnz"])
    An = csr_to_dense(Hn)
    assert rel_fro(oracle_mod.spmm(Hn, X), An @ X) < 1e-14
    assert rel_fro(oracle_mod.spmm_t(Hn, X), An.T @ X) < 1e-14


# --------------------------------------------------------------------------- Rayleigh-Ritz


def test_rayleigh_ritz_full_space_is_brute_force_eigh(oracle_mod):
    H, A, _, _ = _small_case(g=6, w=2)
    N = A.shape[0]
    Y = np.random.default_rng(1).standard_normal((N, N))
    theta, Psi, XF = oracle_mod.rayleigh_ritz(H, Y)
    lam = np.linalg.eigvalsh(A)
    assert np.max(np.abs(theta - lam)) < 1e-12 * np.max(np.abs(lam))
    assert np.max(np.abs(XF.T @ XF - np.eye(N))) < 1e-13
    assert rel_fro(A @ Psi, Psi * theta) < 1e-12


def test_rayleigh_ritz_subspace_and_interlacing(oracle_mod):
    H, A, X, (a, b, a0) = _small_case(g=8, w=2, n=12)
    Y = oracle_mod.filter(H, X, 8, a, b, a0)
    theta, Psi, XF = oracle_mod.rayleigh_ritz(H, Y)
    # the projected problem built another way: SVD-based orthonormal basis, dense H
    U = scipy.linalg.orth(Y)
    ref = np.linalg.eigvalsh(U.T @ A @ U)
    assert np.max(np.abs(theta - ref)) < 1e-12 * np.max(np.abs(ref))
    lam = np.linalg.eigvalsh(A)
    assert np.all(theta >= lam[: theta.size] - 1e-12)          # Cauchy interlacing
    assert np.max(np.abs(XF.T @ XF - np.eye(XF.shape[1]))) < 1e-13
    assert np.max(np.abs(Psi.T @ Psi - np.eye(Psi.shape[1]))) < 1e-13
    # Ritz vectors satisfy the projected eigen-equation: X_F^T (H Psi - Psi Theta) = 0
    assert np.max(np.abs(XF.T @ (A @ Psi - Psi * theta))) < 1e-12 * np.max(np.abs(lam))


def test_repeated_cycles_converge_to_brute_force(oracle_mod):
    """Algorithm 1 applied repeatedly (Psi -> X, Zhou-Saad bound updates): the
    filter and the Rayleigh-Ritz closure together converge to eigvalsh."""
    g, w, n, m = 10, 2, 48, 10
    H = W.csr_grid(g, w, 0.1, 7)
    lam = np.linalg.eigvalsh(csr_to_dense(H))
    X = W.start_block(H["N"], n, 7)
    a, b, a0 = oracle_mod.lanczos_bounds(H, W.lanczos_start(H["N"], 7), 20, n)
    for _ in range(9):
        theta, X, _ = oracle_mod.rayleigh_ritz(H, oracle_mod.filter(H, X, m, a, b, a0))
        a0, a = theta[0], theta[-1]
    assert np.max(np.abs(theta[:36] - lam[:36]) / np.abs(lam[:36])) <= 1e-12


# --------------------------------------------------------------------------- Lanczos


def test_lanczos_full_space_reproduces_spectrum(oracle_mod):
    d = np.array([3.0, -1.0, 0.5, 7.25, 2.0, 4.5, -0.25, 6.0, 1.0, 5.5])
    H = dense_to_csr(np.diag(d), keep_zeros=False)
    v0 = np.random.default_rng(2).standard_normal(d.size)
    a, b, a0 = oracle_mod.lanczos_bounds(H, v0, 20, 2)
    assert abs(a0 - d.min()) < 1e-12 and abs(b - d.max()) < 1e-11
    assert abs(a - (a0 + (b - a0) * (2 / 10) ** (2 / 3))) < 1e-12


def test_lanczos_relation_and_bounds(oracle_mod):
    H, A, _, _ = _small_case(g=8, w=2)
    N = A.shape[0]
    v0 = W.lanczos_start(N, 77)
    al, be, V = oracle_mod.lanczos(H, v0, 20, return_basis=True)
    k = al.size
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    assert np.max(np.abs(V @ V.T - np.eye(k))) < 1e-13
    assert np.max(np.abs(V @ A @ V.T - T)) < 1e-12
    lam = np.linalg.eigvalsh(A)
    a, b, a0 = oracle_mod.lanczos_bounds(H, v0, 20, 32)
    assert b >= lam[-1] - 1e-12                   # upper bound safeguard holds
    assert a0 >= lam[0] - 1e-12                   # Ritz values interlace
    assert a0 - lam[0] < 0.05 * (lam[-1] - lam[0])
    assert a0 < a < b


# --------------------------------------------------------------------------- adjoint


def _loss_grad(Y, w):
    return 2.0 * w[:, None] * Y


def test_adjoint_dX_is_filter_of_G(oracle_mod):
    """p(H) is symmetric, so dX = p(H)^T G = p(H) G (the filter applied to G)."""
    H, _, X, (a, b, a0) = _small_case(g=8, w=2, n=5)
    m = 7
    wts = W.loss_weights(H["N"], 5)
    G = _loss_grad(oracle_mod.filter(H, X, m, a, b, a0), wts)
    dX, _ = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    assert rel_fro(dX, oracle_mod.filter(H, G, m, a, b, a0)) < 1e-12


def _complex_filter_loss(A, X, m, a, b, a0, wts):
    """L = sum_i w_i sum_j Y_m[i,j]^2 (analytic) with Y_m = T_m(t(A)) X / T_m(tau),
    T_m evaluated by the unscaled three-term Chebyshev recurrence (complex A)."""
    e, c = (b - a) / 2.0, (b + a) / 2.0
    tau = (a0 - c) / e
    tA = (A - c * np.eye(A.shape[0])) / e
    Zp, Z = X.astype(complex), tA @ X
    for _ in range(2, m + 1):
        Zp, Z = Z, 2.0 * (tA @ Z) - Zp
    Tm_tau = cheb_T(m, np.array([tau]))[0]
    Y = (Z if m >= 1 else Zp) / Tm_tau
    return np.sum(wts[:, None] * Y * Y)


def test_adjoint_dH_complex_step(oracle_mod):
    H, A, X, (a, b, a0) = _small_case(g=4, w=1, n=3, seed=12)
    m = 6
    wts = W.loss_weights(H["N"], 6)
    G = _loss_grad(oracle_mod.filter(H, X, m, a, b, a0), wts)
    _, dH = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    rows = np.repeat(np.arange(H["N"]), np.diff(H["row_ptr"]))
    h = 1e-30
    picks = np.random.default_rng(0).choice(H["nnz"], 60, replace=False)
    for p in picks:
        Ac = A.astype(complex)
        Ac[rows[p], H["col"][p]] += 1j * h
        cs = np.imag(_complex_filter_loss(Ac, X, m, a, b, a0, wts)) / h
        assert abs(cs - dH[p]) <= 1e-11 * max(1.0, np.max(np.abs(dH)))


def test_adjoint_dH_daleckii_krein(oracle_mod):
    """dL/dH = Q (P o (Q^T G X^T Q)) Q^T, P_ij = divided differences of p."""
    H, A, X, (a, b, a0) = _small_case(g=6, w=2, n=4, seed=13)
    m = 9
    wts = W.loss_weights(H["N"], 7)
    Y = oracle_mod.filter(H, X, m, a, b, a0)
    G = _loss_grad(Y, wts)
    _, dH = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    lam, Q = np.linalg.eigh(A)
    pl = p_of(lam, m, a, b, a0)
    dl = lam[:, None] - lam[None, :]
    close = np.abs(dl) < 1e-7
    P = np.where(close, 0.0, (pl[:, None] - pl[None, :]) / np.where(close, 1.0, dl))
    dpl = dp_of(lam, m, a, b, a0)
    P = np.where(close, 0.5 * (dpl[:, None] + dpl[None, :]), P)
    Dfull = Q @ (P * (Q.T @ G @ X.T @ Q)) @ Q.T
    rows = np.repeat(np.arange(H["N"]), np.diff(H["row_ptr"]))
    ref = Dfull[rows, H["col"]]
    assert np.max(np.abs(dH - ref)) < 1e-9 * np.max(np.abs(ref))


def test_adjoint_dH_central_differences(oracle_mod):
    H, _, X, (a, b, a0) = _small_case(g=6, w=2, n=4, seed=14)
    m = 8
    wts = W.loss_weights(H["N"], 8)

    def loss(val):
        Hp = dict(H)
        Hp["val"] = val
        Y = oracle_mod.filter(Hp, X, m, a, b, a0)
        s = np.sum(wts[:, None] * Y * Y, axis=1)
        return math.fsum(s)

    G = _loss_grad(oracle_mod.filter(H, X, m, a, b, a0), wts)
    _, dH = oracle_mod.filter_adjoint(H, X, m, a, b, a0, G)
    step = 1e-6
    scale = np.max(np.abs(dH))
    for p in np.random.default_rng(1).choice(H["nnz"], 25, replace=False):
        vp, vm = H["val"].copy(), H["val"].copy()
        vp[p] += step
        vm[p] -= step
        fd = (loss(vp) - loss(vm)) / (2 * step)
        # "1e-6 relative" read as relative to the gradient's largest entry
        assert abs(fd - dH[p]) <= 1e-6 * scale


# --------------------------------------------------------------------------- generator


@pytest.mark.parametrize("g,w", [(5, 1), (6, 2), (9, 3), (20, 2), (32, 2), (12, 4)])
def test_generator_nnz_closed_form_and_symmetry(g, w):
    H = W.csr_grid(g, w, 0.1, 9)
    assert H["nnz"] == (g * (2 * w + 1) - w * (w + 1)) ** 3
    if g <= 12:
        A = csr_to_dense(H)
        assert np.array_equal(A, A.T)
        # columns ascending within each row
        for r in range(0, H["N"], 37):
            c = H["col"][H["row_ptr"][r]:H["row_ptr"][r + 1]]
            assert np.all(np.diff(c) > 0)


def test_generator_kinetic_part_is_spd_kronecker_sum():
    g, w = 7, 2
    H0 = csr_to_dense(W.csr_grid(g, w, 0.0, 1))
    A = np.zeros((g, g))
    for i in range(g):
        for j in range(g):
            d = abs(i - j)
            A[i, j] = 2.5 if d == 0 else (-1.0 / (1 + d) ** 2 if d <= w else 0.0)
    I = np.eye(g)
    K = np.kron(np.kron(A, I), I) + np.kron(np.kron(I, A), I) + np.kron(np.kron(I, I), A)
    assert np.array_equal(H0, K)
    assert np.linalg.eigvalsh(K)[0] > 0


def test_generator_blocked_layout_is_a_permutation():
    g, w = 8, 3
    H = W.csr_grid(g, w, 0.1, 2, core_frac=0.1, core_shift=2.0)
    B = W.bsr_from_csr(H, g)
    perm = B["perm"]
    assert np.array_equal(np.sort(perm), np.arange(g ** 3))
    A = csr_to_dense(H)[np.ix_(perm, perm)]
    Ab = np.zeros_like(A)
    bd = B["bdim"]
    for br in range(B["n_block_rows"]):
        for q in range(B["brow_ptr"][br], B["brow_ptr"][br + 1]):
            bc = B["bcol"][q]
            Ab[br * bd:(br + 1) * bd, bc * bd:(bc + 1) * bd] = B["val"][q * bd * bd:(q + 1) * bd * bd].reshape(bd, bd)
    assert np.array_equal(A, Ab)
    assert B["n_blocks"] == (3 * (g // 4) - 2) ** 3


def test_generator_is_reproducible():
    a = W.csr_grid(6, 2, 0.1, 42)
    b = W.csr_grid(6, 2, 0.1, 42)
    c = W.csr_grid(6, 2, 0.1, 43)
    assert np.array_equal(a["val"], b["val"]) and not np.array_equal(a["val"], c["val"])
    X = W.start_block(216, 10, 5)
    assert np.max(np.abs(X.T @ X - np.eye(10))) < 1e-14
