"""Failure paths of the C ABI, each provoked on the host: a device-side wait
that gives up, non-finite input values, a zero pivot in a dense leaf.  None
of them faults or hangs the GPU: the executor's waits are bounded, and once
the status word is set every remaining task is skipped and marked done, so
the launch always drains and the context stays usable."""
import numpy as np
import pytest

import hmat_synth as hs
from gpu_util import GpuProblem, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def test_bounded_wait_gives_up_with_timeout_and_the_next_call_succeeds(ctx):
    """spin_limit = 1: the first dependency wait that does not find its
    predecessor finished gives up at once; hmat_lu returns HMAT_ERR_TIMEOUT
    after the launch drained.  A following call with the default limit on a
    fresh copy of the matrix factors it normally."""
    g = hm()
    p = hs.small_laplace(16, 3, 64, 1e-4)  # about 12 000 tasks, long dependency chains
    gp = GpuProblem(ctx, p)
    with pytest.raises(g.HmatError) as ei:
        gp.H.lu(p.eps, spin_limit=1)
    assert ei.value.code == g.HMAT_ERR_TIMEOUT
    assert gp.H.stats()["status"] == g.HMAT_ERR_TIMEOUT
    fresh = GpuProblem(ctx, p, trees_of=gp)
    fresh.H.lu(p.eps)
    assert fresh.H.stats()["status"] == 0
    err = fresh.precond_error(hs.start_vector(p.n, 0)[fresh.perm])
    assert err < 1e-3


def test_nonfinite_input_is_rejected(ctx):
    """A NaN or an Inf among the CSR values: the scatter kernel counts the
    non-finite entries and hmat_create_from_csr returns HMAT_ERR_NONFINITE."""
    g = hm()
    p = hs.small_laplace(8, 2, 8, 0.0)
    ct = g.ClusterTree(ctx, p.coords(), p.leaf)
    bt = g.BlockTree(ctx, ct, ct, p.eta)
    for bad in (np.nan, np.inf):
        csr = p.matrix()
        csr.val[5] = bad
        with pytest.raises(g.HmatError) as ei:
            g.HMatrix(ctx, bt, csr)
        assert ei.value.code == g.HMAT_ERR_NONFINITE
        assert "non-finite" in str(ei.value)


def test_zero_pivot_names_the_dense_leaf(ctx):
    """The first permuted unknown gets a zero diagonal entry: the no-pivot LU
    of the first dense diagonal leaf meets a zero pivot, hmat_lu returns
    HMAT_ERR_SINGULAR and the message names that leaf."""
    g = hm()
    p = hs.small_laplace(8, 2, 8, 0.0)
    csr = p.matrix()
    ct = g.ClusterTree(ctx, p.coords(), p.leaf)
    bt = g.BlockTree(ctx, ct, ct, p.eta)
    r0 = int(ct.perm()[0])
    k = next(e for e in range(csr.rowptr[r0], csr.rowptr[r0 + 1]) if csr.colidx[e] == r0)
    csr.val[k] = 0.0
    H = g.HMatrix(ctx, bt, csr)
    with pytest.raises(g.HmatError) as ei:
        H.lu(0.0)
    assert ei.value.code == g.HMAT_ERR_SINGULAR
    msg = str(ei.value)
    assert "leaf LU" in msg and "dense diagonal leaf, block-tree node" in msg and "permuted rows 0.." in msg
