"""GPU H-LU at the full sizes the bench times, and edge cases: properties
that hold at any size (the oracle does not run at these sizes), checked in
the bench's launch configuration (one schedule, one persistent launch)."""
import numpy as np
import pytest

import hmat_synth as hs
from gpu_util import GpuProblem, from_dev, hm, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def test_laplace3d_32_mixed_matches_plain_fp64(ctx):
    """32^3, leaf 64, eps 1e-4: the chosen (mixed) form and the plain FP64 form,
    which the smaller parity tests pin to the oracle, reach the same
    preconditioner quality on the same block structure.  The mixed form also
    accumulates the small non-leaf blocks densely (one truncation per flush
    instead of one per product), so it runs fewer truncations."""
    g = hm()
    p = hs.laplace3d_32()
    a = GpuProblem(ctx, p)
    b = GpuProblem(ctx, p, csr=a.csr, trees_of=a)
    a.H.lu(p.eps, precision=g.HMAT_FP64)
    b.H.lu(p.eps, precision=g.HMAT_MIXED, reuse_schedule=True)
    sa, sb = a.H.stats(), b.H.stats()
    assert sa["status"] == 0 and sb["status"] == 0
    assert 0 < sb["truncations"] < sa["truncations"]
    assert sb["gang_truncations"] > 0  # the 1024 x 1024 blocks ran as gangs of CTAs
    v0 = hs.start_vector(p.n, 0)
    ea = a.precond_error(v0[a.perm])
    eb = b.precond_error(v0[b.perm])
    assert eb <= 2.0 * ea and ea <= 2.0 * eb
    assert ea <= 2 * p.eps
    ra, rb = a.H.ranks(), b.H.ranks()
    assert np.array_equal(ra >= 0, rb >= 0)
    assert rb[rb >= 0].mean() <= ra[ra >= 0].mean() + 1.0


def test_diffusion_batch_full_size_quality(ctx):
    """The 64-instance diffusion batch (sides 48..128) in one launch, mixed,
    against the plain FP64 batch: the same quality instance by instance."""
    g = hm()
    probs = hs.diffusion2d_batch()
    A = [GpuProblem(ctx, p) for p in probs]
    B = [GpuProblem(ctx, p, csr=a.csr, trees_of=a) for p, a in zip(probs, A)]
    g.lu_batched(ctx, [a.H for a in A], probs[0].eps, precision=g.HMAT_FP64)
    g.lu_batched(ctx, [b.H for b in B], probs[0].eps, precision=g.HMAT_MIXED)
    assert A[0].H.stats()["status"] == 0 and B[0].H.stats()["status"] == 0
    for i in (0, 17, 42, 63):
        v0 = hs.start_vector(probs[i].n, 0)
        ea = A[i].precond_error(v0[A[i].perm])
        eb = B[i].precond_error(v0[B[i].perm])
        assert eb <= 2.0 * ea and ea <= 2.0 * eb, i


def test_single_leaf_problem_is_dense_lu(ctx):
    """n below the leaf size: one dense leaf, the H-LU is the dense LU and the
    solve is exact."""
    p = hs.small_laplace(3, 2, 16, 0.0)
    gp = GpuProblem(ctx, p)
    A = gp.dense()
    gp.H.lu(0.0)
    D = gp.dense()
    n = p.n
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    assert np.abs(L @ U - A).max() <= 1e-13 * np.abs(A).max()
    b = hs.start_vector(n, 1)
    t = to_dev(b)
    gp.H.solve(t)
    assert np.abs(A @ from_dev(t)[:, 0] - b).max() <= 1e-12 * np.abs(b).max()


def test_rank_cap_is_reported(ctx):
    """A rank cap below what the rule needs ends the factorisation with
    HMAT_ERR_RANK (the device status), not with a silent result."""
    g = hm()
    p = hs.small_laplace(16, 2, 8, 1e-12)
    gp = GpuProblem(ctx, p)
    with pytest.raises(g.HmatError) as e:
        gp.H.lu(p.eps, max_rank=1)
    assert e.value.code == g.HMAT_ERR_RANK
