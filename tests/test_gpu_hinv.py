"""GPU H-matrix inversion with accumulated updates (Fig. invert) against the
dense inverse and against the oracle's inversion."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import GpuProblem, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def test_hinv_eps0_is_the_inverse(ctx):
    """eps = 0: the dense inverse of the permuted matrix (LAPACK as the
    independent reference); blocks of at most 64 x 64 keep exact ranks within
    the leaf capacity."""
    p = hs.small_laplace(8, 2, 8, 0.0)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.invert(0.0)
    assert gp.H.stats()["status"] == 0
    Ai = np.linalg.inv(A)
    assert np.abs(gp.dense() - Ai).max() <= 1e-10 * np.abs(Ai).max()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(16, 2, 8), (8, 3, 16)], ids=["2d16", "3d8"])
def test_hinv_truncated_matches_oracle(ctx, shape, precision):
    """eps = 1e-4: ||I - Hinv A||_2 within 2x of the oracle's inversion of the
    same matrix; the same block structure and (FP64) ranks within 2."""
    N, d, leaf = shape
    p = hs.small_laplace(N, d, leaf, 1e-4)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.invert(p.eps, precision=precision)
    assert gp.H.stats()["status"] == 0
    err_gpu = np.linalg.norm(np.eye(p.n) - gp.dense() @ A, 2)
    ct, bt, csr, H = oracle.setup(p)
    Ao = H.to_dense()
    assert np.array_equal(Ao, A)
    H.invert(p.eps)
    err_orc = np.linalg.norm(np.eye(p.n) - H.to_dense() @ Ao, 2)
    assert err_gpu <= 2.0 * err_orc and err_orc <= 2.0 * err_gpu
    rg, ro = gp.H.ranks(), H.ranks()
    assert np.array_equal(rg >= 0, ro >= 0)
    adm = rg >= 0
    if precision == 0:
        assert np.abs(rg[adm] - ro[adm]).max() <= 2
    else:
        assert rg[adm].mean() <= ro[adm].mean() + 1.0
