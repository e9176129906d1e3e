"""GPU truncation kernel (Section 3 "Truncation", Fig. rkadd) vs the oracle,
element by element on the reconstructed products and singular values."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import from_dev, hm, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


CASES = [(60, 45, 12, 1e-3), (30, 80, 20, 1e-6), (64, 64, 70, 1e-4), (5, 90, 8, 1e-2), (100, 100, 16, 0.0),
         (64, 64, 128, 1e-4), (513, 257, 40, 1e-5), (2000, 1500, 30, 1e-4), (1, 1, 1, 0.0), (7, 3, 9, 0.0)]


@pytest.mark.parametrize("m,n,ell,eps", CASES)
def test_trunc_matches_oracle(ctx, m, n, ell, eps):
    A, B = hs.lowrank_stack(m, n, ell, seed=m * 7 + n + ell, decay=0.6)
    Co, Do = oracle.trunc(A, B, eps)
    U, V = to_dev(A), to_dev(B)
    k = hm().trunc_lowrank(ctx, U, V, eps)
    C, D = from_dev(U, k), from_dev(V, k)
    R = A @ B.T
    nrm = np.linalg.norm(R)
    s = np.linalg.svd(R, compute_uv=False)
    ko = Co.shape[1]
    # ranks equal unless a singular value sits on the threshold
    if k != ko:
        tail_k = np.sqrt(np.sum(s[min(k, ko):] ** 2))
        assert abs(k - ko) == 1 and abs(tail_k - eps * nrm) <= 1e-8 * nrm
    # products equal to rounding (relative to the matrix), same optimal error
    assert np.linalg.norm(C @ D.T - Co @ Do.T) <= 1e-11 * nrm + (s[min(k, ko)] if k != ko else 0)
    assert np.linalg.norm(R - C @ D.T) <= np.sqrt(np.sum(s[k:] ** 2)) * (1 + 1e-6) + 1e-12 * nrm
    # left factor orthonormal (Fig. rkadd: C = U(:, 1:k))
    assert np.allclose(C.T @ C, np.eye(k), atol=1e-10)


def test_trunc_rank_deficient_and_zero(ctx):
    A, B = hs.lowrank_stack(50, 40, 16, seed=9, decay=0.2, deficient=5)
    U, V = to_dev(A), to_dev(B)
    k = hm().trunc_lowrank(ctx, U, V, 0.0)
    R = A @ B.T
    assert np.abs(from_dev(U, k) @ from_dev(V, k).T - R).max() <= 1e-12 * np.abs(R).max()
    U, V = to_dev(np.zeros((10, 3))), to_dev(np.zeros((7, 3)))
    assert hm().trunc_lowrank(ctx, U, V, 1e-4) == 0


def test_trunc_batched(ctx):
    import torch
    g = hm()
    sizes = [(64, 64, 70), (128, 300, 20), (33, 17, 5), (64, 512, 64), (900, 64, 40)]
    Us, Vs, ref = [], [], []
    for i, (m, n, l) in enumerate(sizes):
        A, B = hs.lowrank_stack(m, n, l, seed=100 + i, decay=0.4)
        Us.append(to_dev(A))
        Vs.append(to_dev(B))
        ref.append(oracle.trunc(A, B, 1e-5))
    kn = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    g.trunc_lowrank_batched(ctx, Us, Vs, 1e-5, kn)
    kn = kn.cpu().numpy()
    for i, (Co, Do) in enumerate(ref):
        k = int(kn[i])
        assert abs(k - Co.shape[1]) <= 1
        P = from_dev(Us[i], k) @ from_dev(Vs[i], k).T
        assert np.linalg.norm(P - Co @ Do.T) <= 1e-5 * np.linalg.norm(Co @ Do.T) * 2


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_trunc_batched_mixed_meets_rule(ctx, eps):
    """Randomised range finder (FP32 sketch, FP64 core): the result meets the
    relative Frobenius rule, and its rank is the optimal rank or a little more."""
    import torch
    g = hm()
    sizes = [(64, 64, 70), (64, 128, 72), (128, 300, 20), (33, 17, 12), (200, 64, 40), (512, 512, 24)]
    Us, Vs, data = [], [], []
    for i, (m, n, l) in enumerate(sizes):
        A, B = hs.lowrank_stack(m, n, l, seed=300 + i, decay=0.35)
        Us.append(to_dev(A))
        Vs.append(to_dev(B))
        data.append((A, B))
    kn = torch.zeros(len(sizes), dtype=torch.int64, device="cuda")
    nr = g.trunc_lowrank_batched(ctx, Us, Vs, eps, kn, precision=g.HMAT_MIXED)
    assert nr >= len(sizes) - 1
    kn = kn.cpu().numpy()
    for i, (A, B) in enumerate(data):
        k = int(kn[i])
        R = A @ B.T
        s = np.linalg.svd(R, compute_uv=False)
        kopt = int(np.searchsorted(-np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]), -eps * np.linalg.norm(R)))
        C, D = from_dev(Us[i], k), from_dev(Vs[i], k)
        assert np.all(np.isfinite(C)) and np.all(np.isfinite(D))
        err = np.linalg.norm(R - C @ D.T)
        assert err <= eps * np.linalg.norm(R) * (1 + 1e-3)
        assert kopt - 1 <= k <= kopt + 3
        assert np.allclose(C.T @ C, np.eye(k), atol=1e-5)
