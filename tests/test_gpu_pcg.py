"""hmat_pcg: conjugate gradients preconditioned by the H-LU factors (the
solve check of the stress workload) against the oracle's PCG with its own
factors of the same matrix: the same iteration counts and solutions."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import GpuProblem, hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return hm().Context(0)


def _rhs(n, count, seed=4):
    return np.stack([hs.normal(seed + c, n) for c in range(count)], axis=1)  # n x count, original ordering


def _run_gpu(gp, B, rtol=1e-10):
    import torch
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.zeros_like(Bt)
    its, res = gp.H.pcg(gp.csr, Bt, Xt, rtol=rtol)
    return Xt.cpu().numpy().T, its, res


def test_pcg_exact_factors_one_step(ctx):
    p = hs.small_laplace(16, 2, 8, 0.0)
    gp = GpuProblem(ctx, p)
    gp.H.lu(0.0)
    B = _rhs(p.n, 3)
    X, its, res = _run_gpu(gp, B)
    assert np.all(its <= 2) and np.all(res <= 1e-10)
    assert np.abs(gp.csr.to_dense() @ X - B).max() <= 1e-9 * np.abs(B).max()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_pcg_matches_oracle_iterations(ctx, precision):
    """A variable-coefficient diffusion problem, factors at eps 1e-3: the
    GPU's PCG needs the oracle's iteration count (FP64: within one step;
    mixed: within two) and reaches the same solution."""
    p = hs.Problem("diffusion2d_48", 48, 2, 16, 2.0, 1e-3, kind="diffusion", lc=0.1, seed=11)
    gp = GpuProblem(ctx, p)
    gp.H.lu(p.eps, precision=precision)
    B = _rhs(p.n, 4)
    X, its, res = _run_gpu(gp, B)
    ct, bt, csr, OH = oracle.setup(p)
    OH.lu(p.eps, True)
    Xo, its_o, res_o = OH.pcg(csr, B, rtol=1e-10)
    assert np.all(res <= 1e-9) and np.all(res_o <= 1e-9)
    tol_it = 1 if precision == 0 else 2
    assert np.all(np.abs(its - its_o) <= tol_it), (its, its_o)
    assert np.abs(X - Xo).max() <= 1e-7 * np.abs(Xo).max()
