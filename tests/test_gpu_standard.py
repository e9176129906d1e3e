"""The standard (non-accumulated) form on the GPU (hmat_opts.mode =
HMAT_STANDARD): every product of a leaf pair applied at once by rkupdate
(Section 4, the multiplication before "Accumulated updates", and the remark
after the complexity theorem), and the relative spectral rank rule.  Both
against dense linear algebra and against the oracle's standard form."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import GpuProblem, assert_matches_oracle, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def dense_lu_nopivot(A):
    M = A.copy()
    for k in range(M.shape[0]):
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
    return M


@pytest.mark.parametrize("N,d,leaf", [(16, 2, 8), (8, 3, 16), (24, 2, 32)])
def test_standard_lu_eps0_is_dense_lu(ctx, N, d, leaf):
    g = hm()
    p = hs.small_laplace(N, d, leaf, 0.0)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.lu(0.0, mode=g.HMAT_STANDARD)
    ref = dense_lu_nopivot(A)
    assert np.abs(gp.dense() - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("N,d,leaf,eps", [(16, 2, 8, 1e-4), (8, 3, 16, 1e-4)])
def test_standard_lu_matches_the_oracles_standard_form(ctx, N, d, leaf, eps):
    """FP64: the same rkupdates in the same order as the oracle's standard
    H-LU, so the same ranks and the same factors entry by entry; the standard
    form truncates more often than the accumulated one (Section 4)."""
    g = hm()
    p = hs.small_laplace(N, d, leaf, eps)
    gp = GpuProblem(ctx, p)
    gp.H.lu(eps, mode=g.HMAT_STANDARD)
    t_std = gp.H.stats()["truncations"]
    ct, bt, csr, OH = oracle.setup(p)
    OH.lu(eps, accumulated=False)
    assert_matches_oracle(gp, OH)
    acc = GpuProblem(ctx, p, trees_of=gp)
    acc.H.lu(eps)
    assert acc.H.stats()["truncations"] < t_std


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_standard_lu_quality_against_oracle(ctx, precision):
    """A larger 3D case: preconditioner error within 2x of the oracle's
    standard form, and of the GPU's accumulated form (the paper finds the two
    forms of comparable accuracy)."""
    g = hm()
    p = hs.small_laplace(16, 3, 64, 1e-4)
    gp = GpuProblem(ctx, p)
    gp.H.lu(p.eps, precision=precision, mode=g.HMAT_STANDARD)
    assert gp.H.stats()["status"] == 0
    v0 = hs.start_vector(p.n, 0)
    err = gp.precond_error(v0[gp.perm])
    ct, bt, csr, OH = oracle.setup(p)
    OH.lu(p.eps, accumulated=False)
    err_o, _ = OH.precond_error(csr, v0)
    assert err <= 2.0 * err_o and err_o <= 2.0 * err


def test_standard_addmul_exact_and_matches_oracle(ctx):
    """hmat_addmul in the standard form: exact at eps 0 (Z + alpha X Y) and at
    eps 1e-4 as accurate as the oracle's standard multiplication."""
    g = hm()
    p = hs.small_laplace(16, 2, 8, 1e-6)
    X = GpuProblem(ctx, p)
    X.H.lu(1e-6)
    Z = GpuProblem(ctx, p, csr=X.csr, trees_of=X)
    Dx, Dz = X.dense(), Z.dense()
    g.addmul(ctx, -1.0, X.H, X.H, Z.H, 0.0, mode=g.HMAT_STANDARD)
    ref = Dz - Dx @ Dx
    assert np.abs(Z.dense() - ref).max() <= 1e-12 * (np.abs(Dz).max() + (np.abs(Dx) @ np.abs(Dx)).max())
    # eps > 0: relative spectral error of the product against the oracle's
    Z2 = GpuProblem(ctx, p, csr=X.csr, trees_of=X)
    g.addmul(ctx, -1.0, X.H, X.H, Z2.H, 1e-4, mode=g.HMAT_STANDARD)
    e_gpu = np.linalg.norm(Z2.dense() - ref, 2) / np.linalg.norm(ref, 2)
    ct, bt, csr, OX = oracle.setup(p)
    OX.lu(1e-6, True)
    OZ = oracle.HMatrix.from_csr(bt, csr)
    oracle.hmul(-1.0, OX, OX, OZ, 1e-4, accumulated=False)
    e_orc = np.linalg.norm(OZ.to_dense() - ref, 2) / np.linalg.norm(ref, 2)
    assert e_gpu <= 2.0 * e_orc + 1e-12 and e_orc <= 2.0 * e_gpu + 1e-12


def test_spectral_rank_rule_matches_the_oracle(ctx):
    """rank_rule = HMAT_REL_SPEC (FP64): every truncation keeps the singular
    values above eps sigma_1; the factors equal the oracle's under the same
    rule.  The mixed form refuses the rule."""
    g = hm()
    p = hs.small_laplace(16, 2, 8, 1e-4)
    gp = GpuProblem(ctx, p)
    gp.H.lu(p.eps, rank_rule=g.HMAT_REL_SPEC)
    ct, bt, csr, OH = oracle.setup(p)
    oracle.set_rank_rule(1)
    try:
        OH.lu(p.eps, True)
    finally:
        oracle.set_rank_rule(0)
    assert_matches_oracle(gp, OH)
    with pytest.raises(g.HmatError) as ei:
        GpuProblem(ctx, p, trees_of=gp).H.lu(p.eps, precision=g.HMAT_MIXED, rank_rule=g.HMAT_REL_SPEC)
    assert ei.value.code == g.HMAT_ERR_ARG
