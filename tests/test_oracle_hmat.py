"""Pins of the oracle's H-matrix arithmetic against dense linear algebra
(numpy/LAPACK) and the structural facts of Sections 3-6."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle


def random_hmatrix(bt, seed, k=3):
    """H-matrix on bt with random dense leaves and random rank-k leaves
    (inputs drawn from the seeded generator)."""
    H = oracle.HMatrix.zero(bt)
    bn = bt.nodes()
    cn = bt.rows.nodes()
    off = 0
    for b in range(len(bn["t"])):
        m, n = int(cn["size"][bn["t"][b]]), int(cn["size"][bn["s"][b]])
        if bn["kind"][b] == 1:
            H.set_dense(b, hs.normal(seed, m * n, off).reshape(n, m).T)
            off += m * n
        elif bn["kind"][b] == 2:
            A = hs.normal(seed, m * k, off).reshape(k, m).T
            off += m * k
            B = hs.normal(seed, n * k, off).reshape(k, n).T * 0.3
            off += n * k
            H.set_lowrank(b, A, B)
    return H


def trees(N, d, leaf, eta=2.0):
    ct = oracle.ClusterTree(hs.grid_coords(N, d), leaf)
    return ct, oracle.BlockTree(ct, ct, eta)


def test_from_csr_roundtrip():
    p = hs.small_laplace(16, 2, 8, 0.0)
    ct, bt, csr, H = oracle.setup(p)
    perm = ct.perm()
    assert np.array_equal(H.to_dense(), csr.to_dense()[np.ix_(perm, perm)])
    assert np.all(H.ranks()[bt.nodes()["kind"] == 2] == 0)


@pytest.mark.parametrize("N,d,leaf", [(16, 2, 8), (8, 3, 16)])
def test_addeval_matches_dense(N, d, leaf):
    ct, bt = trees(N, d, leaf)
    H = random_hmatrix(bt, 11)
    G = H.to_dense()
    X = hs.normal(3, G.shape[0] * 4).reshape(-1, 4)
    Y0 = hs.normal(4, G.shape[0] * 4).reshape(-1, 4)
    assert np.allclose(H.addeval(0.5, X, Y0), Y0 + 0.5 * G @ X, atol=1e-12 * np.abs(G).max() * G.shape[0])
    assert np.allclose(H.addeval(-2.0, X, Y0, trans=True), Y0 - 2.0 * G.T @ X,
                       atol=1e-12 * np.abs(G).max() * G.shape[0])


def product_tree_size(bt):
    """#T_IJK from eq. (product_block): (t,s,r) in T_IJK iff (t,s) in T_IJ and
    (s,r) in T_JK (here all three trees are the same)."""
    bn = bt.nodes()
    by_row = np.bincount(bn["t"], minlength=bn["t"].max() + 1)
    return int(sum(by_row[s] for s in bn["s"]))


@pytest.mark.parametrize("accumulated", [False, True])
def test_hmul_exact_at_eps0(accumulated):
    ct, bt = trees(16, 2, 8)
    X, Y, Z = random_hmatrix(bt, 1), random_hmatrix(bt, 2), random_hmatrix(bt, 3)
    Xd, Yd, Zd = X.to_dense(), Y.to_dense(), Z.to_dense()
    oracle.stats_reset()
    oracle.hmul(-0.5, X, Y, Z, 0.0, accumulated)
    ref = Zd - 0.5 * Xd @ Yd
    assert np.abs(Z.to_dense() - ref).max() <= 1e-12 * np.abs(ref).max()
    st = oracle.stats()
    if accumulated:
        # every node of the product tree is visited exactly once
        assert st["addproducts"] + st["pending"] == product_tree_size(bt)


def test_hmul_truncated_error_and_modes_agree():
    ct, bt = trees(32, 2, 8)
    X, Y = random_hmatrix(bt, 5, k=2), random_hmatrix(bt, 6, k=2)
    Xd, Yd = X.to_dense(), Y.to_dense()
    ref = Xd @ Yd
    nrm = np.linalg.norm(ref, 2)
    res = {}
    for acc in (False, True):
        Z = oracle.HMatrix.zero(bt)
        oracle.hmul(1.0, X, Y, Z, 1e-4, acc)
        res[acc] = Z.to_dense()
        # relative spectral error well below the truncation tolerance scale
        assert np.linalg.norm(res[acc] - ref, 2) / nrm < 1e-3
    assert np.linalg.norm(res[True] - res[False], 2) / nrm < 1e-3


def dense_lu_nopivot(A):
    M = A.copy()
    for k in range(M.shape[0]):
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
    return M


@pytest.mark.parametrize("N,d,leaf", [(32, 2, 16), (16, 2, 8), (8, 3, 16), (10, 3, 32)])
@pytest.mark.parametrize("accumulated", [False, True])
def test_hlu_eps0_is_dense_lu(N, d, leaf, accumulated):
    p = hs.small_laplace(N, d, leaf, 0.0)
    ct, bt, csr, H = oracle.setup(p)
    perm = ct.perm()
    A = csr.to_dense()[np.ix_(perm, perm)]
    H.lu(0.0, accumulated)
    D = H.to_dense()
    n = A.shape[0]
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    # L unit lower, U upper with L U = P A P^T determine the no-pivot LU
    assert np.abs(L @ U - A).max() <= 1e-12 * np.abs(A).max()
    assert np.abs(D - dense_lu_nopivot(A)).max() <= 1e-10 * np.abs(D).max()
    # solves with the factors
    b = hs.normal(8, n * 2).reshape(n, 2)
    x = H.solve(b)
    assert np.abs(A @ x - b).max() <= 1e-10 * np.abs(b).max()
    y = H.solve(b, trans=True)
    assert np.abs(A.T @ y - b).max() <= 1e-10 * np.abs(b).max()


def precond_error_dense(D, A):
    n = A.shape[0]
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    E = np.eye(n) - np.linalg.solve(U, np.linalg.solve(L, A))
    return np.linalg.norm(E, 2)


@pytest.mark.parametrize("N,d,leaf,eps", [(32, 2, 16, 1e-3), (10, 3, 32, 1e-2)])
def test_precond_error_power_iteration(N, d, leaf, eps):
    p = hs.small_laplace(N, d, leaf, eps)
    ct, bt, csr, H = oracle.setup(p)
    perm = ct.perm()
    A = csr.to_dense()[np.ix_(perm, perm)]
    H.lu(eps, True)
    exact = precond_error_dense(H.to_dense(), A)
    est, it = H.precond_error(csr, hs.start_vector(p.n, 0)[perm], maxit=200, rtol=1e-6)
    assert 0 < exact < 1
    # power iteration converges to the largest singular value from below
    assert est <= exact * (1 + 1e-9) and est >= 0.9 * exact


def test_accumulated_fewer_truncations_same_quality():
    p = hs.laplace2d_64()
    res = {}
    for acc in (False, True):
        ct, bt, csr, H = oracle.setup(p)
        oracle.stats_reset()
        H.lu(p.eps, acc)
        st = oracle.stats()
        err, _ = H.precond_error(csr, hs.start_vector(p.n, 0))
        res[acc] = (st["truncations"], st["flops_trunc"], err)
    assert res[True][0] < res[False][0] and res[True][1] < res[False][1]
    assert res[True][2] < 2 * res[False][2] + 1e-12
    assert res[True][2] < 1e-4


# ---------------------------------------------------------------------------
# H-matrix inversion with accumulated updates (Fig. invert)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,d,leaf", [(16, 2, 8), (8, 3, 16)])
def test_hinv_eps0_is_the_inverse(N, d, leaf):
    """eps = 0 keeps every non-zero singular value: the result is the inverse
    of the permuted matrix (LAPACK's, as an independent reference)."""
    p = hs.small_laplace(N, d, leaf, 0.0)
    ct, bt, csr, H = oracle.setup(p)
    A = H.to_dense()
    H.invert(0.0)
    Ai = np.linalg.inv(A)
    assert np.abs(H.to_dense() - Ai).max() <= 1e-12 * np.abs(Ai).max()


def test_hinv_diagonal_matrix_exact_at_any_eps():
    """A diagonal matrix: every off-diagonal product is zero, so the
    accumulated updates vanish and the inverse is exact whatever eps."""
    p = hs.small_laplace(16, 2, 8, 1e-2)
    x = p.coords()
    ct = oracle.ClusterTree(x, p.leaf)
    bt = oracle.BlockTree(ct, ct, p.eta)
    n = p.n
    diag = 1.0 + hs.uniform(5, n)
    csr = hs.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int64), diag)
    H = oracle.HMatrix.from_csr(bt, csr)
    H.invert(1e-2)
    perm = ct.perm()
    assert np.allclose(H.to_dense(), np.diag(1.0 / diag[perm]), rtol=1e-14, atol=0.0)


def test_hinv_error_follows_eps():
    """eps > 0: ||I - Hinv A||_2 is of the order of eps and falls with it."""
    p = hs.small_laplace(16, 2, 8, 1e-4)
    errs = []
    for eps in (1e-4, 1e-6):
        ct, bt, csr, H = oracle.setup(p)
        A = H.to_dense()
        H.invert(eps)
        errs.append(np.linalg.norm(np.eye(p.n) - H.to_dense() @ A, 2))
    assert errs[0] <= 1e-2 and errs[1] <= errs[0] / 20


# ---------------------------------------------------------------------------
# H-Cholesky with accumulated updates (Section 6, treated like the inversion)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prob", ["laplace2d_16", "laplace3d_8", "diffusion2d_20"])
def test_hchol_eps0_is_the_cholesky_factor(prob):
    """eps = 0: the lower blocks hold LAPACK's Cholesky factor of the permuted
    SPD matrix."""
    p = {"laplace2d_16": hs.small_laplace(16, 2, 8, 0.0), "laplace3d_8": hs.small_laplace(8, 3, 16, 0.0),
         "diffusion2d_20": hs.Problem("diffusion2d_20", 20, 2, 8, 2.0, 0.0, kind="diffusion", lc=0.1, seed=7)}[prob]
    ct, bt, csr, H = oracle.setup(p)
    A = H.to_dense()
    H.cholesky(0.0)
    Lr = np.linalg.cholesky(A)
    assert np.abs(np.tril(H.to_dense()) - Lr).max() <= 1e-12 * np.abs(Lr).max()


def test_hchol_error_follows_eps_and_halves_the_truncations():
    """eps > 0: ||I - (L L^T)^{-1} A||_2 of the order of eps and falling with it;
    the symmetric recursion truncates about half as often as the LU."""
    p = hs.small_laplace(16, 2, 8, 1e-4)
    errs = []
    for eps in (1e-4, 1e-6):
        ct, bt, csr, H = oracle.setup(p)
        A = H.to_dense()
        oracle.stats_reset()
        H.cholesky(eps)
        tc = oracle.stats()["truncations"]
        L = np.tril(H.to_dense())
        errs.append(np.linalg.norm(np.eye(p.n) - np.linalg.solve(L @ L.T, A), 2))
    assert errs[0] <= 10 * 1e-4 and errs[1] <= errs[0] / 20
    ct, bt, csr, H = oracle.setup(p)
    oracle.stats_reset()
    H.lu(1e-6, True)
    tl = oracle.stats()["truncations"]
    assert 0.4 * tl <= tc <= 0.6 * tl


def test_hinv_standard_and_accumulated_agree():
    """The standard inversion (every product applied at once) and the
    accumulated one (Fig. invert) agree to O(eps), reach errors within a small
    factor of each other, and the accumulated one truncates less often."""
    p = hs.small_laplace(16, 2, 8, 1e-4)
    out = {}
    for acc in (True, False):
        ct, bt, csr, H = oracle.setup(p)
        A = H.to_dense()
        oracle.stats_reset()
        H.invert(p.eps, accumulated=acc)
        D = H.to_dense()
        out[acc] = (D, np.linalg.norm(np.eye(p.n) - D @ A, 2), oracle.stats()["truncations"])
    Ai = np.linalg.inv(A)
    assert np.linalg.norm(out[True][0] - out[False][0], 2) <= 10 * p.eps * np.linalg.norm(Ai, 2)
    assert out[True][1] <= 4 * out[False][1] and out[False][1] <= 4 * out[True][1]
    assert out[True][2] < out[False][2]


# ---------------------------------------------------------------------------
# The reading "dense accumulators for blocks with a leaf cluster" against the
# literal low-rank accumulators of Section 4 (rkadd per addproduct leaf case)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,d,leaf", [(16, 2, 8), (8, 3, 16)])
def test_literal_accumulators_exact_at_eps0(N, d, leaf):
    """With eps = 0 the literal form loses nothing either: its H-LU is the
    dense no-pivot LU of the permuted matrix."""
    p = hs.small_laplace(N, d, leaf, 0.0)
    ct, bt, csr, H = oracle.setup(p)
    A = H.to_dense()
    H.lu(0.0, True, literal=True)
    ref = dense_lu_nopivot(A)
    assert np.abs(H.to_dense() - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("N,d,leaf,eps", [(32, 2, 8, 1e-4), (8, 3, 16, 1e-4), (16, 2, 8, 1e-6)])
def test_literal_accumulators_agree_with_dense_reading_lu(N, d, leaf, eps):
    """Both accumulator forms represent the same sum (Section 4); they differ
    by the truncations the literal one runs per product.  So the factors agree
    to O(eps) and both preconditioner errors are O(eps).  The dense reading
    replaces those truncations by exact sums: it truncates less often than the
    literal form (and than the standard algorithm) and its error is no larger
    than the literal form's (measured: 1.7x to 19x smaller on these grids) and
    equal to the standard algorithm's within 1.5x."""
    p = hs.small_laplace(N, d, leaf, eps)
    out = {}
    for mode in ("dense", "literal", "standard"):
        ct, bt, csr, H = oracle.setup(p)
        A = H.to_dense()
        oracle.stats_reset()
        H.lu(eps, mode != "standard", literal=mode == "literal")
        out[mode] = (H.to_dense(), precond_error_dense(H.to_dense(), A), oracle.stats()["truncations"])
    D0, e0, t0 = out["dense"]
    D1, e1, t1 = out["literal"]
    Ds, es, ts = out["standard"]
    assert np.linalg.norm(D1 - D0, 2) <= 100 * eps * np.linalg.norm(D0, 2)
    assert e0 <= 100 * eps and e1 <= 100 * eps
    assert e0 <= 1.05 * e1
    assert e0 <= 1.5 * es and es <= 1.5 * e0
    assert t0 < ts < t1


def test_literal_accumulators_agree_with_dense_reading_hmul():
    """The same comparison for Z <- Z + X Y: both within O(eps) of the dense
    product and of each other; the literal form truncates more often."""
    ct, bt = trees(32, 2, 8)
    X, Y = random_hmatrix(bt, 5, k=2), random_hmatrix(bt, 6, k=2)
    ref = X.to_dense() @ Y.to_dense()
    nrm = np.linalg.norm(ref, 2)
    res, tr = {}, {}
    for literal in (False, True):
        Z = oracle.HMatrix.zero(bt)
        oracle.stats_reset()
        oracle.hmul(1.0, X, Y, Z, 1e-4, True, literal=literal)
        tr[literal] = oracle.stats()["truncations"]
        res[literal] = Z.to_dense()
        assert np.linalg.norm(res[literal] - ref, 2) / nrm < 1e-3
    assert np.linalg.norm(res[True] - res[False], 2) / nrm < 1e-3
    assert tr[True] > tr[False]


# ---------------------------------------------------------------------------
# Preconditioned CG with the H-LU factors (the PCG check of the stress case)
# ---------------------------------------------------------------------------
def test_pcg_with_exact_factors_converges_in_one_step():
    """With eps = 0 the preconditioner is A^{-1}: one CG step solves A x = b
    to rounding (the residual of the exact solve)."""
    p = hs.small_laplace(16, 2, 8, 0.0)
    ct, bt, csr, H = oracle.setup(p)
    H.lu(0.0, True)
    B = np.stack([hs.normal(4 + c, p.n) for c in range(3)], axis=1)
    X, its, res = H.pcg(csr, B, rtol=1e-10)
    assert np.all(its <= 2) and np.all(res <= 1e-10)
    A = csr.to_dense()
    assert np.abs(A @ X - B).max() <= 1e-9 * np.abs(B).max()


def test_pcg_iterations_fall_with_eps():
    """A diffusion problem: the H-LU preconditioner at a tighter eps needs
    fewer CG iterations to the same residual, and every run reaches it."""
    p = hs.Problem("diffusion2d_32", 32, 2, 16, 2.0, 1e-2, kind="diffusion", lc=0.1, seed=11)
    B = np.stack([hs.normal(40 + c, p.n) for c in range(2)], axis=1)
    its = {}
    for eps in (1e-1, 1e-3):
        ct, bt, csr, H = oracle.setup(p)
        H.lu(eps, True)
        X, it, res = H.pcg(csr, B, rtol=1e-10)
        assert np.all(res <= 1e-9)
        its[eps] = int(it.max())
    assert its[1e-3] < its[1e-1]
