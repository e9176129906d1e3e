"""GPU H-Cholesky with accumulated updates against LAPACK's Cholesky factor
and against the oracle's H-Cholesky."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import GpuProblem, assert_matches_oracle, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def test_hchol_eps0_is_the_cholesky_factor(ctx):
    p = hs.small_laplace(8, 2, 8, 0.0)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.cholesky(0.0)
    assert gp.H.stats()["status"] == 0
    Lr = np.linalg.cholesky(A)
    D = gp.dense()
    assert np.abs(np.tril(D) - Lr).max() <= 1e-10 * np.abs(Lr).max()
    # the upper blocks and upper triangles of the diagonal leaves hold L^T
    assert np.abs(np.triu(D) - Lr.T).max() <= 1e-10 * np.abs(Lr).max()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(16, 2, 8), (8, 3, 16)], ids=["2d16", "3d8"])
def test_hchol_truncated_matches_oracle(ctx, shape, precision):
    N, d, leaf = shape
    p = hs.small_laplace(N, d, leaf, 1e-4)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.cholesky(p.eps, precision=precision)
    assert gp.H.stats()["status"] == 0
    L = np.tril(gp.dense())
    err_gpu = np.linalg.norm(np.eye(p.n) - np.linalg.solve(L @ L.T, A), 2)
    ct, bt, csr, H = oracle.setup(p)
    H.cholesky(p.eps)
    Lo = np.tril(H.to_dense())
    err_orc = np.linalg.norm(np.eye(p.n) - np.linalg.solve(Lo @ Lo.T, A), 2)
    assert err_gpu <= 2.0 * err_orc and err_orc <= 2.0 * err_gpu
    if precision == 0:
        # FP64: the same truncations in the same order up to rounding, so the
        # factor agrees with the oracle's entry by entry, L^T above included
        assert_matches_oracle(gp, H)
