"""Input generators: determinism and the properties of the stand-in workloads."""
import math

import numpy as np

import hmat_synth as hs


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (Steele, Lea, Flood 2014; also the seeding routine of xoshiro).
    x = hs.splitmix64(0, 3)
    assert [int(v) for v in x] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_normal_moments():
    u = hs.uniform(5, 200000)
    assert 0.0 < u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005
    z = hs.normal(6, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert np.array_equal(hs.normal(6, 10), hs.normal(6, 10))


def test_laplacian_structure():
    for N, d in [(7, 2), (5, 3)]:
        A = hs.laplacian(N, d).to_dense()
        assert np.array_equal(A, A.T)
        assert np.all(np.diag(A) == 2 * d)
        off = A - np.diag(np.diag(A))
        assert set(np.unique(off)) <= {0.0, -1.0}
        # rows of interior points sum to zero; boundary rows are positive
        x = hs.grid_coords(N, d)
        h = 1.0 / (N + 1)
        interior = np.all((x > 1.5 * h) & (x < 1 - 1.5 * h), axis=1)
        rs = A.sum(axis=1)
        assert np.allclose(rs[interior], 0.0) and np.all(rs[~interior] > 0)
        # smallest eigenvalue of the h^2-scaled 5/7-point Laplacian
        lam = np.linalg.eigvalsh(A).min()
        assert abs(lam - d * 2 * (1 - math.cos(math.pi * h))) < 1e-10


def test_diffusion_symmetric_and_row_sums():
    f = hs.rff_field(2, 0.1, seed=3, M=256)
    csr = hs.diffusion(12, 2, f)
    A = csr.to_dense()
    assert np.allclose(A, A.T)
    assert np.all(np.diag(A) > 0) and np.all(A - np.diag(np.diag(A)) <= 0)
    assert np.all(A.sum(axis=1) > -1e-12)
    assert np.linalg.eigvalsh(A).min() > 0


def test_rff_covariance():
    # Stationary field with unit variance and squared-exponential covariance
    # exp(-r^2 / (2 lc^2)), checked empirically within Monte-Carlo error.
    lc = 0.1
    pts = np.array([[0.3, 0.3], [0.37, 0.3]])
    r2 = float(np.sum((pts[0] - pts[1]) ** 2))
    vals = np.array([hs.rff_field(2, lc, seed=s, M=512)(pts) for s in range(1500)])
    var = vals.var(axis=0)
    cov = np.mean(vals[:, 0] * vals[:, 1]) - vals[:, 0].mean() * vals[:, 1].mean()
    assert np.all(np.abs(var - 1.0) < 0.12)
    assert abs(cov - math.exp(-r2 / (2 * lc * lc))) < 0.12


def test_batch_sides():
    probs = hs.diffusion2d_batch()
    sides = [p.N for p in probs]
    assert len(sides) == 64 and min(sides) >= 48 and max(sides) <= 128
    assert sides == [p.N for p in hs.diffusion2d_batch()]
