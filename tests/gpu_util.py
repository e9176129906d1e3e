"""Helpers of the GPU parity tests (marshalling only)."""
import numpy as np


def hm():
    from paper_1703_09085_gb300 import build
    build.build()
    import paper_1703_09085_gb300 as g
    return g


def to_dev(a: np.ndarray):
    """n x k column-major numpy matrix -> CUDA tensor (k, n)."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def from_dev(t, ncol=None) -> np.ndarray:
    a = t.cpu().numpy().T
    return a if ncol is None else a[:, :ncol]


class GpuProblem:
    """Trees, H-matrix and CSR of a synthetic problem on the GPU path."""

    def __init__(self, ctx, problem, csr=None, trees_of=None):
        g = hm()
        self.p = problem
        self.csr = csr if csr is not None else problem.matrix()
        if trees_of is not None:  # share the cluster and block trees of another problem
            self.ct, self.bt = trees_of.ct, trees_of.bt
        else:
            self.ct = g.ClusterTree(ctx, problem.coords(), problem.leaf)
            self.bt = g.BlockTree(ctx, self.ct, self.ct, problem.eta)
        self.H = g.HMatrix(ctx, self.bt, self.csr)
        self.perm = self.ct.perm()

    def dense(self) -> np.ndarray:
        import torch
        n = self.csr.n
        out = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        self.H.to_dense(out)
        return out.cpu().numpy().T

    def precond_error(self, v0, maxit=50, rtol=1e-3):
        """||I - (LU)^{-1} A||_2 by power iteration on E^T E (same recipe as the
        oracle's), with the GPU solves and a CPU sparse product."""
        perm = self.perm
        A = self.csr

        def Ap(v):  # permuted A times v
            x = np.zeros(A.n)
            x[perm] = v
            y = A.matvec(x)
            return y[perm]

        v = v0 / np.linalg.norm(v0)
        est = 0.0
        for it in range(maxit):
            w = Ap(v)
            t = to_dev(w)
            self.H.solve(t)
            w = v - from_dev(t)[:, 0]
            new = np.linalg.norm(w)
            t = to_dev(w)
            self.H.solve(t, trans=True)
            z = w - Ap(from_dev(t)[:, 0])  # A symmetric: A^T = A
            done = it > 0 and abs(new - est) <= rtol * new
            est = new
            nz = np.linalg.norm(z)
            if nz == 0:
                break
            v = z / nz
            if done:
                break
        return est


def assert_matches_oracle(gp: GpuProblem, OH, rtol: float = 1e-10):
    """The FP64 GPU result equals the oracle's entry by entry: every admissible
    block has the oracle's rank (the block trees are the same, so the rank
    vectors line up node by node) and the dense matrices agree to rtol
    relative to the largest entry."""
    rg = gp.H.ranks()
    ro = OH.ranks()
    assert rg.shape == ro.shape
    diff = np.flatnonzero(rg != ro)
    assert diff.size == 0, f"{diff.size} blocks differ in rank from the oracle (first {diff[:5]})"
    D = gp.dense()
    Do = OH.to_dense()
    scale = np.abs(Do).max()
    err = np.abs(D - Do).max()
    assert err <= rtol * scale, f"max entry difference {err / scale:.3e} relative"
