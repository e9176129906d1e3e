"""Seeded synthetic inputs for the H-LU hot path.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_1703_09085_gb300``).  It produces *inputs only*: grid
coordinates, finite-difference matrices in CSR form, random fields, random
factor stacks and random start vectors.  It holds none of the method's
arithmetic (no trees, no truncation, no factorisation).

The paper measures on boundary-element matrices built by hybrid cross
approximation (Section 7).  Those are not reproducible here; the stand-in
workloads are finite-difference Laplacians and variable-coefficient diffusion
operators on the unit square/cube with Dirichlet boundary conditions, whose
H-matrix blocks far from the diagonal start at rank zero (Section 3, opening
paragraph: stiffness matrices of differential operators have local rank 0).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw ``i`` of stream ``seed`` is ``mix64(seed + (i+1)*GAMMA)``.
Normals come from the Box-Muller transform.  Everything is vectorised numpy
with wrapping uint64 arithmetic, so the same seed gives the same bits on x86
and Arm.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` raw 64-bit draws of stream ``seed`` starting at draw ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        return _mix64(s + i * GAMMA)


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    x = splitmix64(seed, count, offset) >> np.uint64(11)
    return (x.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles by Box-Muller on consecutive uniform pairs."""
    npair = (count + 1) // 2
    u = uniform(seed, 2 * npair, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npair)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def randint(seed: int, lo: int, hi: int, count: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by rejection-free scaling."""
    u = uniform(seed, count)
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)


# ---------------------------------------------------------------------------
# Grids and finite-difference operators
# ---------------------------------------------------------------------------

def grid_coords(N: int, d: int) -> np.ndarray:
    """Interior points of the uniform grid with N points per direction on the
    unit square (d=2) or cube (d=3), h = 1/(N+1), lexicographic order with x
    fastest.  Returns an (N**d, d) float64 array, row-major."""
    h = 1.0 / (N + 1)
    ax = (np.arange(N, dtype=np.float64) + 1.0) * h
    if d == 2:
        y, x = np.meshgrid(ax, ax, indexing="ij")
        return np.stack([x.ravel(), y.ravel()], axis=1)
    if d == 3:
        z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    raise ValueError("d must be 2 or 3")


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64, n+1
    colidx: np.ndarray  # int64, nnz
    val: np.ndarray     # float64, nnz

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.colidx] = self.val
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        y = np.zeros((self.n,) + x.shape[1:])
        np.add.at(y, rows, self.val.reshape((-1,) + (1,) * (x.ndim - 1)) * x[self.colidx])
        return y


def _assemble(N: int, d: int, face_coeff) -> CSR:
    """Assemble the h^2-scaled 2d+1 point operator -div(k grad u) with
    Dirichlet boundary eliminated.  ``face_coeff(p, axis, sign)`` returns the
    coefficient on the face between point p and its neighbour p + sign*e_axis
    (for a neighbour on the boundary, the face between p and the boundary
    point)."""
    n = N ** d
    idx = np.arange(n, dtype=np.int64)
    sub = [(idx // (N ** a)) % N for a in range(d)]
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for a in range(d):
        for sign in (-1, 1):
            c = face_coeff(idx, a, sign)
            diag += c
            inside = (sub[a] + sign >= 0) & (sub[a] + sign < N)
            rows.append(idx[inside])
            cols.append(idx[inside] + sign * (N ** a))
            vals.append(-c[inside])
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr, c.astype(np.int64), v.astype(np.float64))


def laplacian(N: int, d: int) -> CSR:
    """5-point (d=2) or 7-point (d=3) Laplacian scaled by h^2: diagonal 2d,
    off-diagonal -1 to interior neighbours."""
    return _assemble(N, d, lambda p, a, s: np.ones(p.shape[0]))


@dataclasses.dataclass
class RFFField:
    """g(x) = sqrt(2/M) * sum_j cos(w_j . x + phi_j) with w_j ~ N(0, lc^-2 I),
    phi_j ~ U[0, 2 pi): a random-Fourier-feature realisation of a stationary
    Gaussian field with squared-exponential covariance exp(-|x-y|^2/(2 lc^2))
    and unit variance (Rahimi and Recht, NIPS 2007)."""
    omega: np.ndarray  # (M, d)
    phi: np.ndarray    # (M,)

    def __call__(self, x: np.ndarray, chunk: int = 16384) -> np.ndarray:
        M = self.phi.shape[0]
        out = np.empty(x.shape[0])
        for i in range(0, x.shape[0], chunk):
            arg = x[i:i + chunk] @ self.omega.T + self.phi
            out[i:i + chunk] = np.cos(arg).sum(axis=1)
        return out * math.sqrt(2.0 / M)


    def grid(self, axes) -> np.ndarray:
        """g on the tensor grid axes[0] x axes[1] (x ...), axis 0 fastest, as a
        flat array.  cos(w.x + phi) = Re(e^{i phi} prod_a e^{i w_a x_a}), so the
        grid of values is a complex matrix product over the M features."""
        M = self.phi.shape[0]
        E = [np.exp(1j * np.outer(self.omega[:, a], ax)) for a, ax in enumerate(axes)]  # (M, n_a)
        w = np.exp(1j * self.phi)
        if len(axes) == 2:
            G = ((E[0] * w[:, None]).T @ E[1]).real  # (n0, n1)
            return G.T.ravel() * math.sqrt(2.0 / M)
        out = np.empty((len(axes[2]), len(axes[1]), len(axes[0])))
        for k in range(len(axes[2])):
            G = ((E[0] * (w * E[2][:, k])[:, None]).T @ E[1]).real
            out[k] = G.T
        return out.ravel() * math.sqrt(2.0 / M)


def rff_field(d: int, lc: float, seed: int, M: int = 2048) -> RFFField:
    omega = normal(seed, M * d).reshape(M, d) / lc
    phi = 2.0 * math.pi * uniform(seed ^ 0x5A5A5A5A, M)
    return RFFField(omega, phi)


def diffusion(N: int, d: int, field: RFFField) -> CSR:
    """-div(k grad u) with k = exp(g), g a seeded field; face coefficients are
    k at the face midpoints (between a point and its neighbour, or the boundary
    point).  Scaled by h^2.  Each of the (N+1) N^(d-1) faces per axis is
    evaluated once: face f along an axis sits at (f + 1/2) h."""
    h = 1.0 / (N + 1)
    ax = (np.arange(N, dtype=np.float64) + 1.0) * h
    fx = (np.arange(N + 1, dtype=np.float64) + 0.5) * h
    kf = []
    for a in range(d):
        axes = [fx if b == a else ax for b in range(d)]
        kf.append(np.exp(field.grid(axes)))  # lexicographic, axis 0 fastest

    def coeff(p, a, s):
        sub = [(p // (N ** b)) % N for b in range(d)]
        f = sub[a] + (1 if s > 0 else 0)
        stride = 1
        idx = np.zeros_like(p)
        for b in range(d):
            idx += (f if b == a else sub[b]) * stride
            stride *= (N + 1) if b == a else N
        return kf[a][idx]

    return _assemble(N, d, coeff)


# ---------------------------------------------------------------------------
# Workload descriptors (the five configurations of the benchmark plan)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    N: int
    d: int
    leaf: int
    eta: float
    eps: float
    kind: str = "laplace"      # or "diffusion"
    lc: float = 0.1
    seed: int = 0

    @property
    def n(self) -> int:
        return self.N ** self.d

    def coords(self) -> np.ndarray:
        return grid_coords(self.N, self.d)

    def matrix(self) -> CSR:
        if self.kind == "laplace":
            return laplacian(self.N, self.d)
        return diffusion(self.N, self.d, rff_field(self.d, self.lc, self.seed))


def laplace2d_64() -> Problem:
    """2D 5-point Laplacian, 64 x 64 interior grid (n = 4096), leaf 32, eta 2, eps 1e-6."""
    return Problem("laplace2d_64", 64, 2, 32, 2.0, 1e-6)


def laplace3d_32() -> Problem:
    """3D 7-point Laplacian, 32^3 grid (n = 32768), leaf 64, eta 2, eps 1e-4."""
    return Problem("laplace3d_32", 32, 3, 64, 2.0, 1e-4)


def laplace3d_64() -> Problem:
    """3D 7-point Laplacian, 64^3 grid (n = 262144), leaf 64, eta 2, eps 1e-4."""
    return Problem("laplace3d_64", 64, 3, 64, 2.0, 1e-4)


def diffusion2d_batch(count: int = 64, seed: int = 2) -> list[Problem]:
    """``count`` independent 2D diffusion problems with grid sides uniform in
    48..128, k = exp(g), g with correlation length 0.1; leaf 32, eps 1e-5.
    Instance i uses field seed ``seed + i``."""
    sides = randint(seed, 48, 128, count)
    return [Problem(f"diffusion2d_{i}", int(sides[i]), 2, 32, 2.0, 1e-5,
                    kind="diffusion", lc=0.1, seed=seed + i) for i in range(count)]


def diffusion3d_80(eps: float = 1e-3) -> Problem:
    """3D diffusion on an 80^3 grid (n = 512000), correlation length 0.05, leaf 64."""
    return Problem("diffusion3d_80", 80, 3, 64, 2.0, eps, kind="diffusion", lc=0.05, seed=4)


def small_laplace(N: int, d: int, leaf: int, eps: float) -> Problem:
    return Problem(f"laplace{d}d_{N}", N, d, leaf, 2.0, eps)


# ---------------------------------------------------------------------------
# Random factor stacks for the truncation kernels
# ---------------------------------------------------------------------------

def lowrank_stack(m: int, n: int, ell: int, seed: int, decay: float = 0.5,
                  deficient: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Factors A (m x ell) and B (n x ell), column-major-friendly float64 arrays,
    with column scales decaying like 10**(-decay*j) so that the product has a
    graded spectrum.  The last ``deficient`` columns of B repeat earlier ones,
    making the stack exactly rank deficient."""
    A = normal(seed, m * ell).reshape(ell, m).T.copy()
    B = normal(seed + 7919, n * ell).reshape(ell, n).T.copy()
    scale = 10.0 ** (-decay * np.arange(ell))
    A *= scale
    for j in range(deficient):
        if ell - 1 - j > 0:
            B[:, ell - 1 - j] = B[:, j % max(1, ell - deficient)]
    return A, B


def start_vector(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) start vector for the power iteration."""
    return normal(seed, n)
