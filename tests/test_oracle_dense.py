"""Pins of the oracle's dense building blocks and of the truncation
(Section 3, "Truncation" and Fig. rkadd) against LAPACK (numpy) and the
Eckart-Young theorem -- independent of the oracle's own QR/SVD code."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle


def rnd(m, n, seed):
    return hs.normal(seed, m * n).reshape(n, m).T.copy()


@pytest.mark.parametrize("m,n", [(40, 7), (7, 7), (5, 9), (64, 64), (200, 30)])
def test_qr(m, n):
    A = rnd(m, n, m * 31 + n)
    Q, R = oracle.qr(A)
    q = min(m, n)
    assert np.allclose(Q @ R, A, atol=1e-13 * np.abs(A).max() * max(m, n))
    assert np.allclose(Q.T @ Q, np.eye(q), atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0.0)


def test_qr_rank_deficient_and_badly_scaled():
    A = rnd(30, 6, 3)
    A[:, 3] = A[:, 0] + A[:, 1]
    A[:, 4] *= 1e-180
    A[:, 5] = 0.0
    Q, R = oracle.qr(A)
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(R))
    assert np.allclose(Q @ R, A, atol=1e-13)
    assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-12)


@pytest.mark.parametrize("m,n", [(50, 8), (8, 50), (33, 33), (1, 5), (6, 1)])
def test_svd_matches_lapack(m, n):
    A = rnd(m, n, 7 * m + n)
    U, s, V = oracle.svd(A)
    sref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, sref, rtol=1e-12, atol=1e-13 * sref[0])
    assert np.allclose((U * s) @ V.T, A, atol=1e-12 * sref[0])
    assert np.allclose(V.T @ V, np.eye(min(m, n)), atol=1e-12)


def graded(m, n, ell, seed, decay=0.7, deficient=0):
    return hs.lowrank_stack(m, n, ell, seed, decay=decay, deficient=deficient)


def rule_rank(s, eps):
    """Smallest k with sum_{i>k} s_i^2 <= eps^2 sum s_i^2, by brute force."""
    tot = np.sum(s ** 2)
    for k in range(len(s) + 1):
        if np.sum(s[k:] ** 2) <= eps * eps * tot:
            return k
    return len(s)


@pytest.mark.parametrize("m,n,ell,eps", [(60, 45, 12, 1e-3), (30, 80, 20, 1e-6), (64, 64, 70, 1e-4),
                                          (5, 90, 8, 1e-2), (100, 100, 16, 0.0)])
def test_truncation_eckart_young(m, n, ell, eps):
    A, B = graded(m, n, ell, seed=m + n + ell)
    C, D = oracle.trunc(A, B, eps)
    R = A @ B.T
    s = np.linalg.svd(R, compute_uv=False)
    k = C.shape[1]
    # optimal error of rank k (Eckart-Young) in the Frobenius norm
    err = np.linalg.norm(R - C @ D.T)
    opt = np.sqrt(np.sum(s[k:] ** 2))
    assert err <= opt * (1 + 1e-6) + 1e-12 * s[0]
    # k is the smallest rank meeting the rule (ties within rounding allowed)
    if eps > 0:
        kr = rule_rank(s, eps)
        assert abs(k - kr) <= 1
        assert err <= eps * np.linalg.norm(R) * (1 + 1e-8) + 1e-13 * s[0]
    else:
        assert err <= 1e-12 * s[0]
    # C has orthonormal columns (Fig. rkadd: C = U(:, 1:k))
    assert np.allclose(C.T @ C, np.eye(k), atol=1e-10)


def test_truncation_rank_deficient_stack():
    A, B = graded(50, 40, 16, seed=9, decay=0.2, deficient=5)
    C, D = oracle.trunc(A, B, 0.0)
    R = A @ B.T
    assert np.allclose(C @ D.T, R, atol=1e-12 * np.abs(R).max())
    assert C.shape[1] <= 16


def test_truncation_zero_and_empty():
    C, D = oracle.trunc(np.zeros((10, 3)), np.zeros((7, 3)), 1e-4)
    assert C.shape == (10, 0) and D.shape == (7, 0)
    C, D = oracle.trunc(np.zeros((10, 0)), np.zeros((7, 0)), 1e-4)
    assert C.shape[1] == 0


@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_rkadd_is_truncated_sum(eps):
    A, B = graded(40, 35, 6, seed=1)
    C, D = graded(40, 35, 5, seed=2)
    Co, Do = oracle.rkadd(-0.75, A, B, C, D, eps)
    S = C @ D.T - 0.75 * A @ B.T
    s = np.linalg.svd(S, compute_uv=False)
    k = Co.shape[1]
    err = np.linalg.norm(S - Co @ Do.T)
    assert err <= np.sqrt(np.sum(s[k:] ** 2)) * (1 + 1e-6) + 1e-12 * s[0]
    if eps == 0.0:
        assert err <= 1e-12 * s[0]


@pytest.mark.parametrize("m,n,ell,eps", [(40, 30, 12, 1e-3), (25, 60, 20, 1e-6), (16, 16, 16, 0.0)])
def test_spectral_rank_rule_is_eckart_young_in_the_2_norm(m, n, ell, eps):
    """Rank rule 1 (relative spectral): the truncation keeps the smallest k
    with sigma_{k+1} <= eps sigma_1, and the error in the spectral norm is
    exactly sigma_{k+1} (Eckart-Young), against LAPACK's singular values."""
    A, B = hs.lowrank_stack(m, n, ell, seed=31 + m, decay=0.4)
    R = A @ B.T
    s = np.linalg.svd(R, compute_uv=False)
    oracle.set_rank_rule(1)
    try:
        C, D = oracle.trunc(A, B, eps)
    finally:
        oracle.set_rank_rule(0)
    k = C.shape[1]
    assert k == int(np.sum(s > eps * s[0])) if eps > 0 else k == int(np.sum(s > 1e-13 * s[0]))
    err = np.linalg.norm(R - C @ D.T, 2)
    nxt = s[k] if k < len(s) else 0.0
    assert abs(err - nxt) <= 1e-10 * s[0]
