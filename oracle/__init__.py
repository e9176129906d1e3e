"""CPU oracle for H-matrix arithmetic with accumulated updates (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s ``cpu_baseline`` leg and ``--impl reference`` arm may import it.
It is the plain, serial FP64 statement of the method (``hmat_oracle.cpp``),
written from the paper (Boerm, arXiv:1703.09085, Sections 2-7) and shares no code
with the CUDA path in ``paper_1703_09085_gb300``.

Every function here is ctypes marshalling around ``liboracle.so``; the arithmetic
is all in ``hmat_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmat_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

I64P = ctypes.POINTER(ctypes.c_int64)
F64P = ctypes.POINTER(ctypes.c_double)
I32P = ctypes.POINTER(ctypes.c_int)
VPP = ctypes.POINTER(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


class Stats(ctypes.Structure):
    _fields_ = [("truncations", ctypes.c_int64), ("rkadds", ctypes.c_int64),
                ("rowmerges", ctypes.c_int64), ("addproducts", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("dense_lu", ctypes.c_int64),
                ("flops", ctypes.c_double), ("seconds", ctypes.c_double),
                ("flops_trunc", ctypes.c_double), ("flops_dense", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile liboracle.so (serial, FP64, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
                   "-o", _LIB + ".tmp", _SRC]
            subprocess.check_call(cmd)
            os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_last_error.restype = ctypes.c_char_p
        L.orc_ctree_size.restype = ctypes.c_int64
        L.orc_btree_size.restype = ctypes.c_int64
        L.orc_trace_size.restype = ctypes.c_int64
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {lib().orc_last_error().decode()}")


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray, t=F64P):
    return a.ctypes.data_as(t)


def stats_reset():
    lib().orc_stats_reset()


def set_rank_rule(rule: int):
    """0: relative Frobenius (default), 1: relative spectral (smallest k with
    sigma_{k+1} <= eps sigma_1); applies to every later truncation."""
    lib().orc_set_rank_rule(ctypes.c_int(rule))


def trace_enable(on: bool = True):
    """Record (rows, cols, stacked width, new rank) of every truncation
    (rowmerge SVDs have a negative width)."""
    lib().orc_trace_enable(ctypes.c_int(1 if on else 0))


def trace() -> np.ndarray:
    n = lib().orc_trace_size()
    out = np.zeros(4 * n, np.int64)
    lib().orc_trace_get(_p(out, I64P))
    return out.reshape(n, 4)


def stats() -> dict:
    s = Stats()
    lib().orc_stats_get(ctypes.byref(s))
    return s.as_dict()


# --------------------------------------------------------------------------
# Dense building blocks
# --------------------------------------------------------------------------

def qr(A):
    A = _f64(A)
    m, n = A.shape
    q = min(m, n)
    Q = np.zeros((m, q), order="F")
    R = np.zeros((q, n), order="F")
    _check(lib().orc_qr(ctypes.c_int64(m), ctypes.c_int64(n), _p(A), _p(Q), _p(R)))
    return Q, R


def svd(A):
    A = _f64(A)
    m, n = A.shape
    p = min(m, n)
    U = np.zeros((m, p), order="F")
    s = np.zeros(p)
    V = np.zeros((n, p), order="F")
    _check(lib().orc_svd(ctypes.c_int64(m), ctypes.c_int64(n), _p(A), _p(U), _p(s), _p(V)))
    return U, s, V


def trunc(A, B, eps: float, max_rank: int = -1):
    """Best rank-k approximation C D^T of A B^T (Section 3, "Truncation")."""
    A, B = _f64(A), _f64(B)
    m, l = A.shape
    n = B.shape[0]
    cap = max(1, min(m, n, l))
    C = np.zeros((m, cap), order="F")
    D = np.zeros((n, cap), order="F")
    k = ctypes.c_int64(0)
    _check(lib().orc_trunc(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(l), _p(A), _p(B),
                           ctypes.c_double(eps), ctypes.c_int64(max_rank), _p(C), _p(D), ctypes.byref(k)))
    return C[:, :k.value].copy(), D[:, :k.value].copy()


def rkadd(alpha: float, A, B, C, D, eps: float):
    """Fig. rkadd: trunc(C D^T + alpha A B^T) as factors."""
    A, B, C, D = _f64(A), _f64(B), _f64(C), _f64(D)
    m, n = A.shape[0], B.shape[0]
    cap = max(1, min(m, n, A.shape[1] + C.shape[1]))
    Co = np.zeros((m, cap), order="F")
    Do = np.zeros((n, cap), order="F")
    k = ctypes.c_int64(0)
    _check(lib().orc_rkadd(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_double(alpha),
                           ctypes.c_int64(A.shape[1]), _p(A), _p(B), ctypes.c_int64(C.shape[1]), _p(C), _p(D),
                           ctypes.c_double(eps), _p(Co), _p(Do), ctypes.byref(k)))
    return Co[:, :k.value].copy(), Do[:, :k.value].copy()


# --------------------------------------------------------------------------
# Trees and H-matrices
# --------------------------------------------------------------------------

class ClusterTree:
    def __init__(self, coords: np.ndarray, leaf: int):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.n, self.d = coords.shape
        h = ctypes.c_void_p()
        _check(lib().orc_ctree_build(_p(coords), ctypes.c_int64(self.n), ctypes.c_int(self.d),
                                     ctypes.c_int64(leaf), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ctree_free(self.h)
            self.h = None

    def nodes(self) -> dict:
        c = lib().orc_ctree_size(self.h)
        off = np.zeros(c, np.int64)
        size = np.zeros(c, np.int64)
        level = np.zeros(c, np.int32)
        parent = np.zeros(c, np.int32)
        nsons = np.zeros(c, np.int32)
        lib().orc_ctree_nodes(self.h, _p(off, I64P), _p(size, I64P), _p(level, I32P), _p(parent, I32P),
                              _p(nsons, I32P))
        return dict(off=off, size=size, level=level, parent=parent, nsons=nsons)

    def perm(self) -> np.ndarray:
        p = np.zeros(self.n, np.int64)
        lib().orc_ctree_perm(self.h, _p(p, I64P))
        return p


class BlockTree:
    def __init__(self, rows: ClusterTree, cols: ClusterTree, eta: float):
        self.rows, self.cols = rows, cols
        h = ctypes.c_void_p()
        _check(lib().orc_btree_build(rows.h, cols.h, ctypes.c_double(eta), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_btree_free(self.h)
            self.h = None

    def nodes(self) -> dict:
        c = lib().orc_btree_size(self.h)
        t = np.zeros(c, np.int32)
        s = np.zeros(c, np.int32)
        level = np.zeros(c, np.int32)
        parent = np.zeros(c, np.int32)
        kind = np.zeros(c, np.int32)
        lib().orc_btree_nodes(self.h, _p(t, I32P), _p(s, I32P), _p(level, I32P), _p(parent, I32P),
                              _p(kind, I32P))
        return dict(t=t, s=s, level=level, parent=parent, kind=kind)


NONLEAF, DENSE, LOWRANK = 0, 1, 2


class HMatrix:
    def __init__(self, bt: BlockTree, h):
        self.bt = bt
        self.h = h
        self.nrows = bt.rows.n
        self.ncols = bt.cols.n

    @classmethod
    def from_csr(cls, bt: BlockTree, csr) -> "HMatrix":
        h = ctypes.c_void_p()
        rp = np.ascontiguousarray(csr.rowptr, np.int64)
        ci = np.ascontiguousarray(csr.colidx, np.int64)
        va = np.ascontiguousarray(csr.val, np.float64)
        _check(lib().orc_hmat_from_csr(bt.h, ctypes.c_int64(csr.n), _p(rp, I64P), _p(ci, I64P), _p(va),
                                       ctypes.byref(h)))
        return cls(bt, h)

    @classmethod
    def zero(cls, bt: BlockTree) -> "HMatrix":
        h = ctypes.c_void_p()
        _check(lib().orc_hmat_zero(bt.h, ctypes.byref(h)))
        return cls(bt, h)

    def copy(self) -> "HMatrix":
        h = ctypes.c_void_p()
        _check(lib().orc_hmat_copy(self.h, ctypes.byref(h)))
        return HMatrix(self.bt, h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_hmat_free(self.h)
            self.h = None

    def set_dense(self, b: int, data):
        data = _f64(data)
        _check(lib().orc_hmat_set_dense(self.h, ctypes.c_int(b), _p(data)))

    def set_lowrank(self, b: int, A, B):
        A, B = _f64(A), _f64(B)
        _check(lib().orc_hmat_set_lowrank(self.h, ctypes.c_int(b), ctypes.c_int64(A.shape[1]), _p(A), _p(B)))

    def ranks(self) -> np.ndarray:
        r = np.zeros(lib().orc_btree_size(self.bt.h), np.int64)
        lib().orc_hmat_ranks(self.h, _p(r, I64P))
        return r

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.nrows, self.ncols), order="F")
        _check(lib().orc_hmat_to_dense(self.h, _p(D)))
        return D

    def addeval(self, alpha: float, X, Y, trans: bool = False) -> np.ndarray:
        X = _f64(X if np.ndim(X) == 2 else np.reshape(X, (-1, 1)))
        Y = _f64(Y if np.ndim(Y) == 2 else np.reshape(Y, (-1, 1))).copy(order="F")
        _check(lib().orc_addeval(self.h, ctypes.c_double(alpha), ctypes.c_int64(X.shape[1]), _p(X), _p(Y),
                                 ctypes.c_int(1 if trans else 0)))
        return Y

    def lu(self, eps: float, accumulated: bool = True, literal: bool = False):
        """In place: H-LU, accumulated (Section 6 with the accumulators of
        Section 4) or standard.  literal=True holds every accumulator in
        low-rank form, as Section 4 states it, instead of keeping the blocks
        with a leaf cluster dense."""
        mode = (2 if literal else 1) if accumulated else 0
        _check(lib().orc_hlu(self.h, ctypes.c_double(eps), ctypes.c_int(mode)))

    def cholesky(self, eps: float):
        """In place: H-Cholesky with accumulated updates; the lower blocks hold L
        (A = L L^T), the upper ones L^T."""
        _check(lib().orc_hchol(self.h, ctypes.c_double(eps)))

    def invert(self, eps: float, accumulated: bool = True):
        """In place: the H-matrix inverse with accumulated updates (Fig. invert),
        or by the standard multiplication."""
        _check(lib().orc_hinv(self.h, ctypes.c_double(eps), ctypes.c_int(1 if accumulated else 0)))

    def solve(self, B, trans: bool = False) -> np.ndarray:
        B = _f64(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1))).copy(order="F")
        _check(lib().orc_hsolve(self.h, ctypes.c_int64(B.shape[1]), _p(B), ctypes.c_int(1 if trans else 0)))
        return B

    def pcg(self, csr, B, rtol: float = 1e-10, maxit: int = 500):
        """Preconditioned CG for A X = B (B: n x nrhs, original ordering) with
        these H-LU factors as the preconditioner; returns X, iterations and
        final relative residuals per column."""
        B = _f64(B if np.ndim(B) == 2 else np.reshape(B, (-1, 1)))
        n, nrhs = B.shape
        X = np.zeros((n, nrhs), order="F")
        its = np.zeros(nrhs, np.int64)
        res = np.zeros(nrhs)
        rp = np.ascontiguousarray(csr.rowptr, np.int64)
        ci = np.ascontiguousarray(csr.colidx, np.int64)
        va = np.ascontiguousarray(csr.val, np.float64)
        _check(lib().orc_pcg(self.h, ctypes.c_int64(n), _p(rp, I64P), _p(ci, I64P), _p(va), ctypes.c_int64(nrhs),
                             _p(B), _p(X), ctypes.c_double(rtol), ctypes.c_int64(maxit), _p(its, I64P), _p(res)))
        return X, its, res

    def precond_error(self, csr, v0, maxit: int = 50, rtol: float = 1e-3):
        rp = np.ascontiguousarray(csr.rowptr, np.int64)
        ci = np.ascontiguousarray(csr.colidx, np.int64)
        va = np.ascontiguousarray(csr.val, np.float64)
        v0 = np.ascontiguousarray(v0, np.float64)
        err = ctypes.c_double(0)
        it = ctypes.c_int(0)
        _check(lib().orc_precond_error(self.h, ctypes.c_int64(csr.n), _p(rp, I64P), _p(ci, I64P), _p(va),
                                       _p(v0), ctypes.c_int(maxit), ctypes.c_double(rtol), ctypes.byref(err),
                                       ctypes.byref(it)))
        return err.value, it.value


def hmul(alpha: float, X: HMatrix, Y: HMatrix, Z: HMatrix, eps: float, accumulated: bool = True,
         literal: bool = False):
    """Z <- blocktrunc(Z + alpha X Y) (Section 4); literal as in HMatrix.lu."""
    mode = (2 if literal else 1) if accumulated else 0
    _check(lib().orc_hmul(ctypes.c_double(alpha), X.h, Y.h, Z.h, ctypes.c_double(eps), ctypes.c_int(mode)))


def setup(problem):
    """Trees and H-matrix of a synthetic problem (cluster tree, block tree, A)."""
    coords = problem.coords()
    ct = ClusterTree(coords, problem.leaf)
    bt = BlockTree(ct, ct, problem.eta)
    csr = problem.matrix()
    H = HMatrix.from_csr(bt, csr)
    return ct, bt, csr, H
