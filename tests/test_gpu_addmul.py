"""GPU H-matrix multiplication Z <- blocktrunc(Z + alpha X Y) (accumulated
form) against dense products and against the oracle's accumulated H-mult."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import GpuProblem, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


PROBS = {"2d": lambda: hs.small_laplace(32, 2, 16, 1e-6), "3d": lambda: hs.small_laplace(12, 3, 32, 1e-6)}
# admissible blocks of at most 32 x 32: exact ranks fit the leaf capacity (64)
SMALL = {"2d": lambda: hs.small_laplace(16, 2, 8, 1e-6), "3d": lambda: hs.small_laplace(8, 3, 16, 1e-6)}


def _gpu_factor(ctx, p, eps, trees_of=None):
    gp = GpuProblem(ctx, p, trees_of=trees_of)
    gp.H.lu(eps)
    return gp


@pytest.mark.parametrize("alpha", [-1.0, 0.5])
@pytest.mark.parametrize("prob", sorted(SMALL))
def test_addmul_eps0_is_exact(ctx, prob, alpha):
    """eps = 0: every truncation keeps all non-zero singular values, so the
    result is Z + alpha X Y up to rounding (X, Y with low-rank and dense
    leaves: the factors of a truncated LU)."""
    g = hm()
    p = SMALL[prob]()
    X = _gpu_factor(ctx, p, 1e-6)
    Y = _gpu_factor(ctx, p, 1e-4, trees_of=X)
    Z = GpuProblem(ctx, p, csr=X.csr, trees_of=X)
    Dx, Dy, Dz = X.dense(), Y.dense(), Z.dense()
    g.addmul(ctx, alpha, X.H, Y.H, Z.H, 0.0)
    st = Z.H.stats()
    assert st["status"] == 0 and st["truncations"] > 0
    ref = Dz + alpha * Dx @ Dy
    scale = np.abs(Dz).max() + abs(alpha) * (np.abs(Dx) @ np.abs(Dy)).max()
    assert np.abs(Z.dense() - ref).max() <= 1e-12 * scale
    # X and Y are read only
    assert np.array_equal(X.dense(), Dx) and np.array_equal(Y.dense(), Dy)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("prob", sorted(PROBS))
def test_addmul_truncated_matches_oracle(ctx, prob, precision):
    """eps > 0: the GPU and the oracle, given the same X, Y and Z (to the
    rounding of an LU at eps 1e-9), reach the same accuracy against the exact
    product, and the same ranks up to threshold cases."""
    g = hm()
    p = PROBS[prob]()
    eps = 1e-4
    X = _gpu_factor(ctx, p, 1e-9)
    Z = GpuProblem(ctx, p, csr=X.csr, trees_of=X)
    Dx, Dz = X.dense(), Z.dense()
    ref = Dz - Dx @ Dx
    Y = _gpu_factor(ctx, p, 1e-9, trees_of=X)
    g.addmul(ctx, -1.0, X.H, Y.H, Z.H, eps, precision=precision)
    err_gpu = np.linalg.norm(Z.dense() - ref, 2) / np.linalg.norm(ref, 2)

    ct, bt, csr, Ho = oracle.setup(p)
    Ho.lu(1e-9, True)
    Yo = Ho.copy()
    Zo = oracle.HMatrix.from_csr(bt, csr)
    Dxo = Ho.to_dense()
    assert np.abs(Dxo - Dx).max() <= 1e-6 * np.abs(Dx).max()
    refo = Zo.to_dense() - Dxo @ Dxo
    oracle.hmul(-1.0, Ho, Yo, Zo, eps, accumulated=True)
    err_orc = np.linalg.norm(Zo.to_dense() - refo, 2) / np.linalg.norm(refo, 2)
    # the blockwise relative Frobenius rule keeps the spectral error a small
    # multiple of eps
    assert err_orc <= 10 * eps and err_gpu <= 10 * eps
    assert err_gpu <= 2.0 * err_orc + 1e-12 and err_orc <= 2.0 * err_gpu + 1e-12
    rg, ro = Z.H.ranks(), Zo.ranks()
    assert np.array_equal(rg >= 0, ro >= 0)
    # blocks whose exact value is zero hold only rounding noise, which the
    # relative rule may keep at any rank: compare the others
    cn, bn = ct.nodes(), bt.nodes()
    off, size = cn["off"], cn["size"]
    bnorm = np.array([np.linalg.norm(ref[off[t]:off[t] + size[t], off[u]:off[u] + size[u]])
                      for t, u in zip(bn["t"], bn["s"])])
    adm = (rg >= 0) & (bnorm > 1e-10 * np.linalg.norm(ref))
    assert adm.sum() > 0.5 * (rg >= 0).sum()
    if precision == 0:
        assert np.abs(rg[adm] - ro[adm]).max() <= 2
        assert abs(rg[adm].mean() - ro[adm].mean()) <= 0.1
    else:
        assert rg[adm].mean() <= ro[adm].mean() + 1.0


def test_addmul_rejects_aliasing_and_other_trees(ctx):
    g = hm()
    p = PROBS["2d"]()
    X = GpuProblem(ctx, p)
    Z = GpuProblem(ctx, p, csr=X.csr, trees_of=X)
    with pytest.raises(g.HmatError) as e:
        g.addmul(ctx, 1.0, X.H, Z.H, Z.H, 1e-4)
    assert e.value.code == g.HMAT_ERR_ARG
    W = GpuProblem(ctx, p)  # same points, its own cluster tree
    with pytest.raises(g.HmatError) as e:
        g.addmul(ctx, 1.0, X.H, W.H, Z.H, 1e-4)
    assert e.value.code == g.HMAT_ERR_ARG
