"""GB300 (sm_103a) H-matrix arithmetic with accumulated updates.

Thin ctypes binding of ``libhmat.so`` (C ABI declared in ``include/hmat.h``).
Every function here only marshals arguments; all arithmetic runs in the CUDA
kernels of ``csrc/``.  Device buffers are torch CUDA tensors (float64,
contiguous, column-major by convention: a tensor of shape (ncol, n) holds an
n x ncol column-major matrix) or raw device pointers.

Importing this module loads the shared library; if it has not been built the
import of any entry point raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhmat.so")
_lib = None

I64P = ctypes.POINTER(ctypes.c_int64)
F64P = ctypes.POINTER(ctypes.c_double)
I32P = ctypes.POINTER(ctypes.c_int)

STATUS = {0: "HMAT_OK", 1: "HMAT_ERR_ARG", 2: "HMAT_ERR_NOMEM", 3: "HMAT_ERR_SINGULAR",
          4: "HMAT_ERR_NONFINITE", 5: "HMAT_ERR_RANK", 6: "HMAT_ERR_TIMEOUT", 7: "HMAT_ERR_CUDA",
          9: "HMAT_ERR_INTERNAL"}
HMAT_FP64, HMAT_MIXED = 0, 1
HMAT_ACCUMULATED, HMAT_STANDARD = 0, 1
HMAT_REL_FRO, HMAT_REL_SPEC = 0, 1

for _code, _name in STATUS.items():  # HMAT_OK, HMAT_ERR_ARG, ... as module constants
    globals()[_name] = _code

# Every symbol include/hmat.h declares.
EXPORTS = ["hmat_last_error", "hmat_ctx_create", "hmat_ctx_destroy", "hmat_clustertree_build",
           "hmat_clustertree_perm", "hmat_clustertree_size", "hmat_clustertree_nodes", "hmat_ctree_destroy",
           "hmat_blocktree_build", "hmat_blocktree_size", "hmat_blocktree_nodes", "hmat_btree_destroy",
           "hmat_create_from_csr", "hmat_destroy", "hmat_to_dense", "hmat_addeval", "hmat_lu", "hmat_solve",
           "trunc_lowrank", "trunc_lowrank_batched", "hmat_stats_get", "hmat_ranks", "hmat_copy_values",
           "hmat_analyze_lu", "trunc_lowrank_noalloc", "hmat_lu_batched", "hmat_lu_training_data",
           "hmat_mlp_create", "hmat_mlp_destroy", "hmat_mlp_get_params", "hmat_mlp_set_params", "hmat_mlp_forward",
           "hmat_mlp_grad", "hmat_mlp_train", "hmat_addmul", "hmat_invert", "hmat_cholesky", "hmat_pcg"]
MLP_NPARAM = 4673


class HmatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_rank", ctypes.c_int64), ("precision", ctypes.c_int),
                ("spin_limit", ctypes.c_int64), ("reuse_schedule", ctypes.c_int), ("predictor", ctypes.c_void_p),
                ("record_training", ctypes.c_int), ("seed", ctypes.c_uint64), ("mode", ctypes.c_int),
                ("rank_rule", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("blocks", ctypes.c_int64), ("dense_leaves", ctypes.c_int64),
                ("lowrank_leaves", ctypes.c_int64), ("max_rank", ctypes.c_int64), ("mean_rank", ctypes.c_double),
                ("tasks", ctypes.c_int64), ("truncations", ctypes.c_int64), ("flops", ctypes.c_double),
                ("factor_seconds", ctypes.c_double),
                ("schedule_seconds", ctypes.c_double), ("device_bytes", ctypes.c_int64), ("status", ctypes.c_int),
                ("levels", ctypes.c_int64), ("critical_flops", ctypes.c_double), ("est_flops", ctypes.c_double),
                ("type_seconds", ctypes.c_double * 16), ("type_count", ctypes.c_int64 * 16),
                ("wait_seconds", ctypes.c_double), ("schedule_reused", ctypes.c_int),
                ("rand_truncations", ctypes.c_int64),
                ("rand_fallbacks", ctypes.c_int64), ("sketch_attempts", ctypes.c_int64),
                ("sketch_columns", ctypes.c_int64), ("training_pairs", ctypes.c_int64), ("cp_seconds", ctypes.c_double),
                ("cp_type_seconds", ctypes.c_double * 16), ("cp_type_count", ctypes.c_int64 * 16),
                ("flops32", ctypes.c_double), ("bytes", ctypes.c_double), ("gang_truncations", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            d[f] = list(v) if f in ("type_seconds", "type_count", "cp_type_seconds", "cp_type_count") else v
        return d


def lib():
    """The loaded libhmat.so; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhmat.so is not built: run paper_1703_09085_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        L.hmat_last_error.restype = ctypes.c_size_t
        L.hmat_clustertree_size.restype = ctypes.c_int64
        L.hmat_blocktree_size.restype = ctypes.c_int64
        for name in EXPORTS:
            if name not in ("hmat_last_error", "hmat_clustertree_size", "hmat_blocktree_size"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().hmat_last_error(buf, ctypes.c_size_t(1024))
    return buf.value.decode(errors="replace")


def _check(rc: int):
    if rc != 0:
        raise HmatError(rc, last_error())


def _dptr(x) -> ctypes.c_void_p:
    """Device pointer of a torch CUDA float64 tensor (or an int address)."""
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if not x.is_cuda or x.dtype.__str__() != "torch.float64" or not x.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(x.data_ptr())


def _hp(a: np.ndarray, t):
    return a.ctypes.data_as(t)


class Context:
    """hmat_ctx_create on `device` issuing work on `stream` (torch stream, raw
    cudaStream_t int, or None for the legacy default stream)."""

    def __init__(self, device: int = 0, stream=None):
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        h = ctypes.c_void_p()
        _check(lib().hmat_ctx_create(ctypes.c_int(device), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().hmat_ctx_destroy(self.h)
            self.h = None

    __del__ = close


class ClusterTree:
    def __init__(self, ctx: Context, coords: np.ndarray, leaf: int):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.n, self.d = coords.shape
        h = ctypes.c_void_p()
        _check(lib().hmat_clustertree_build(ctx.h, _hp(coords, F64P), ctypes.c_int64(self.n), ctypes.c_int(self.d),
                                            ctypes.c_int64(leaf), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().hmat_ctree_destroy(self.h)
            self.h = None

    def perm(self) -> np.ndarray:
        p = np.zeros(self.n, np.int64)
        _check(lib().hmat_clustertree_perm(self.h, _hp(p, I64P)))
        return p

    def nodes(self) -> dict:
        c = lib().hmat_clustertree_size(self.h)
        off = np.zeros(c, np.int64)
        size = np.zeros(c, np.int64)
        level = np.zeros(c, np.int32)
        parent = np.zeros(c, np.int32)
        nsons = np.zeros(c, np.int32)
        _check(lib().hmat_clustertree_nodes(self.h, _hp(off, I64P), _hp(size, I64P), _hp(level, I32P),
                                            _hp(parent, I32P), _hp(nsons, I32P)))
        return dict(off=off, size=size, level=level, parent=parent, nsons=nsons)


class BlockTree:
    def __init__(self, ctx: Context, rows: ClusterTree, cols: ClusterTree, eta: float):
        self.rows, self.cols = rows, cols
        h = ctypes.c_void_p()
        _check(lib().hmat_blocktree_build(ctx.h, rows.h, cols.h, ctypes.c_double(eta), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().hmat_btree_destroy(self.h)
            self.h = None

    def nodes(self) -> dict:
        c = lib().hmat_blocktree_size(self.h)
        arrs = [np.zeros(c, np.int32) for _ in range(5)]
        _check(lib().hmat_blocktree_nodes(self.h, *[_hp(a, I32P) for a in arrs]))
        return dict(zip(["t", "s", "level", "parent", "kind"], arrs))


class HMatrix:
    """An H-matrix in device memory (hmat_create_from_csr)."""

    def __init__(self, ctx: Context, bt: BlockTree, csr):
        self.ctx, self.bt = ctx, bt
        self.n = csr.n
        rp = np.ascontiguousarray(csr.rowptr, np.int64)
        ci = np.ascontiguousarray(csr.colidx, np.int64)
        va = np.ascontiguousarray(csr.val, np.float64)
        h = ctypes.c_void_p()
        _check(lib().hmat_create_from_csr(ctx.h, bt.h, ctypes.c_int64(csr.n), _hp(rp, I64P), _hp(ci, I64P),
                                          _hp(va, F64P), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().hmat_destroy(self.h)
            self.h = None

    def copy_values_from(self, src: "HMatrix"):
        _check(lib().hmat_copy_values(self.ctx.h, self.h, src.h))

    def lu(self, eps: float, max_rank: int = 0, precision: int = HMAT_FP64, spin_limit: int = 0,
           reuse_schedule: bool = False, predictor=None, record_training: bool = False, mode: int = HMAT_ACCUMULATED,
           rank_rule: int = HMAT_REL_FRO):
        o = Opts(eps, max_rank, precision, spin_limit, int(reuse_schedule), predictor.h if predictor else None,
                 int(record_training), 0, mode, rank_rule)
        _check(lib().hmat_lu(self.ctx.h, self.h, ctypes.byref(o)))

    def cholesky(self, eps: float, max_rank: int = 0, precision: int = HMAT_FP64, spin_limit: int = 0):
        """In place: H-Cholesky with accumulated updates (hmat_cholesky); lower
        blocks L, upper blocks L^T."""
        o = Opts(eps, max_rank, precision, spin_limit, 0, None, 0)
        _check(lib().hmat_cholesky(self.ctx.h, self.h, ctypes.byref(o)))

    def invert(self, eps: float, max_rank: int = 0, precision: int = HMAT_FP64, spin_limit: int = 0,
               predictor=None):
        """In place: G <- G^{-1} with accumulated updates (hmat_invert)."""
        o = Opts(eps, max_rank, precision, spin_limit, 0, predictor.h if predictor else None, 0)
        _check(lib().hmat_invert(self.ctx.h, self.h, ctypes.byref(o)))

    def to_dense(self, out):
        _check(lib().hmat_to_dense(self.ctx.h, self.h, _dptr(out)))

    def addeval(self, alpha: float, X, Y, trans: bool = False):
        ncol = X.shape[0] if X.dim() == 2 else 1
        _check(lib().hmat_addeval(self.ctx.h, self.h, ctypes.c_double(alpha), ctypes.c_int(int(trans)),
                                  ctypes.c_int64(ncol), _dptr(X), _dptr(Y)))

    def solve(self, B, trans: bool = False):
        nrhs = B.shape[0] if B.dim() == 2 else 1
        _check(lib().hmat_solve(self.ctx.h, self.h, ctypes.c_int(int(trans)), ctypes.c_int64(nrhs), _dptr(B),
                                ctypes.c_int64(self.n)))

    def pcg(self, csr, B, X, rtol: float = 1e-10, maxit: int = 500):
        """hmat_pcg: CG for A X = B (torch tensors (nrhs, n), original ordering)
        preconditioned by these factors; returns (iterations, relative
        residuals) per right-hand side."""
        nrhs = B.shape[0] if B.dim() == 2 else 1
        rp = np.ascontiguousarray(csr.rowptr, np.int64)
        ci = np.ascontiguousarray(csr.colidx, np.int64)
        va = np.ascontiguousarray(csr.val, np.float64)
        its = np.zeros(nrhs, np.int64)
        res = np.zeros(nrhs)
        _check(lib().hmat_pcg(self.ctx.h, self.h, ctypes.c_int64(self.n), _hp(rp, I64P), _hp(ci, I64P), _hp(va, F64P),
                              ctypes.c_int64(nrhs), _dptr(B), _dptr(X), ctypes.c_double(rtol), ctypes.c_int64(maxit),
                              _hp(its, I64P), _hp(res, F64P)))
        return its, res

    def stats(self) -> dict:
        s = Stats()
        _check(lib().hmat_stats_get(self.h, ctypes.byref(s)))
        return s.as_dict()

    def training_data(self):
        """(X, y) pairs recorded by the last lu(record_training=True)."""
        cnt = ctypes.c_int64(0)
        _check(lib().hmat_lu_training_data(self.h, ctypes.c_int64(0), None, None, ctypes.byref(cnt)))
        X = np.zeros((cnt.value, 6), np.float32)
        y = np.zeros(cnt.value, np.float32)
        _check(lib().hmat_lu_training_data(self.h, ctypes.c_int64(cnt.value), _hp(X, ctypes.POINTER(ctypes.c_float)),
                                           _hp(y, ctypes.POINTER(ctypes.c_float)), ctypes.byref(cnt)))
        return X, y

    def ranks(self) -> np.ndarray:
        r = np.zeros(lib().hmat_blocktree_size(self.bt.h), np.int64)
        _check(lib().hmat_ranks(self.h, _hp(r, I64P)))
        return r


def addmul(ctx: Context, alpha: float, X: "HMatrix", Y: "HMatrix", Z: "HMatrix", eps: float, max_rank: int = 0,
           precision: int = HMAT_FP64, spin_limit: int = 0, predictor=None, record_training: bool = False,
           mode: int = HMAT_ACCUMULATED, rank_rule: int = HMAT_REL_FRO):
    """hmat_addmul: Z <- blocktrunc(Z + alpha X Y), accumulated (or standard) form, one launch."""
    o = Opts(eps, max_rank, precision, spin_limit, 0, predictor.h if predictor else None, int(record_training), 0,
             mode, rank_rule)
    _check(lib().hmat_addmul(ctx.h, ctypes.c_double(alpha), X.h, Y.h, Z.h, ctypes.byref(o)))


def lu_batched(ctx: Context, Hs, eps: float, max_rank: int = 0, precision: int = HMAT_FP64, spin_limit: int = 0,
               reuse_schedule: bool = False, predictor=None, record_training: bool = False,
               mode: int = HMAT_ACCUMULATED, rank_rule: int = HMAT_REL_FRO):
    """hmat_lu_batched: factor the HMatrix objects Hs together in one launch."""
    arr = (ctypes.c_void_p * len(Hs))(*[H.h.value for H in Hs])
    o = Opts(eps, max_rank, precision, spin_limit, int(reuse_schedule), predictor.h if predictor else None,
             int(record_training), 0, mode, rank_rule)
    _check(lib().hmat_lu_batched(ctx.h, arr, ctypes.c_int(len(Hs)), ctypes.byref(o)))


def analyze_lu(bt: BlockTree, csr, eps: float = 0.0, max_rank: int = 0) -> dict:
    """Host-only analysis of the H-LU schedule (hmat_analyze_lu)."""
    rp = np.ascontiguousarray(csr.rowptr, np.int64)
    ci = np.ascontiguousarray(csr.colidx, np.int64)
    va = np.ascontiguousarray(csr.val, np.float64)
    o = Opts(eps, max_rank, HMAT_FP64, 0, 0, None, 0)
    s = Stats()
    _check(lib().hmat_analyze_lu(bt.h, ctypes.c_int64(csr.n), _hp(rp, I64P), _hp(ci, I64P), _hp(va, F64P),
                                 ctypes.byref(o), ctypes.byref(s)))
    return s.as_dict()


def trunc_lowrank(ctx: Context, U, V, eps: float) -> int:
    """In-place truncation of U V^T; U: tensor (k, m) holding m x k column-major,
    V: (k, n).  Returns the new rank (first columns hold the result)."""
    k, m = U.shape
    n = V.shape[1]
    kn = ctypes.c_int64(0)
    _check(lib().trunc_lowrank(ctx.h, ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(k), _dptr(U),
                               ctypes.c_int64(max(m, 1)), _dptr(V), ctypes.c_int64(max(n, 1)), ctypes.c_double(eps),
                               ctypes.byref(kn)))
    return kn.value


def trunc_lowrank_noalloc(ctx: Context, U, V, eps: float) -> int:
    """As trunc_lowrank, through the entry point that allocates no memory
    (fixed scratch compiled into the library; see include/hmat.h)."""
    k, m = U.shape
    n = V.shape[1]
    kn = ctypes.c_int64(0)
    _check(lib().trunc_lowrank_noalloc(ctx.h, ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(k), _dptr(U),
                                       ctypes.c_int64(max(m, 1)), _dptr(V), ctypes.c_int64(max(n, 1)),
                                       ctypes.c_double(eps), ctypes.byref(kn)))
    return kn.value


def trunc_lowrank_batched(ctx: Context, Us, Vs, eps: float, k_new, precision: int = HMAT_FP64) -> int:
    """Batched in-place truncation; Us[i]: (k_i, m_i) tensors, Vs[i]: (k_i, n_i),
    k_new: int64 CUDA tensor of len(Us) receiving the new ranks.  Returns how
    many problems the randomised path (precision=HMAT_MIXED) finished."""
    cnt = len(Us)
    m = np.array([u.shape[1] for u in Us], np.int64)
    k = np.array([u.shape[0] for u in Us], np.int64)
    n = np.array([v.shape[1] for v in Vs], np.int64)
    up = (ctypes.c_void_p * cnt)(*[_dptr(u).value for u in Us])
    vp = (ctypes.c_void_p * cnt)(*[_dptr(v).value for v in Vs])
    rnd = ctypes.c_int64(0)
    _check(lib().trunc_lowrank_batched(ctx.h, ctypes.c_int64(cnt), _hp(m, I64P), _hp(n, I64P), _hp(k, I64P), up, vp,
                                       ctypes.c_double(eps), ctypes.c_void_p(k_new.data_ptr()), ctypes.c_int(precision),
                                       ctypes.byref(rnd)))
    return rnd.value


F32P = ctypes.POINTER(ctypes.c_float)


class RankPredictor:
    """The rank predictor (hmat_mlp_*): 3-layer MLP, BF16 weights, FP32
    accumulation, trained on the GPU by the library's own kernels."""

    def __init__(self, ctx: Context, seed: int = 0):
        h = ctypes.c_void_p()
        _check(lib().hmat_mlp_create(ctx.h, ctypes.c_uint64(seed), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().hmat_mlp_destroy(self.h)
            self.h = None

    def params(self) -> np.ndarray:
        p = np.zeros(MLP_NPARAM, np.float32)
        _check(lib().hmat_mlp_get_params(self.h, _hp(p, F32P)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().hmat_mlp_set_params(self.h, _hp(p, F32P)))

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        y = np.zeros(X.shape[0], np.float32)
        _check(lib().hmat_mlp_forward(self.h, ctypes.c_int64(X.shape[0]), _hp(X, F32P), _hp(y, F32P)))
        return y

    def grad(self, X, y):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = ctypes.c_float(0)
        g = np.zeros(MLP_NPARAM, np.float32)
        _check(lib().hmat_mlp_grad(self.h, ctypes.c_int64(X.shape[0]), _hp(X, F32P), _hp(y, F32P), ctypes.byref(loss),
                                   _hp(g, F32P)))
        return loss.value, g

    def train(self, X, y, epochs: int = 30, batch: int = 256, lr: float = 3e-3, seed: int = 3) -> float:
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        loss = ctypes.c_float(0)
        _check(lib().hmat_mlp_train(self.h, ctypes.c_int64(X.shape[0]), _hp(X, F32P), _hp(y, F32P), ctypes.c_int(epochs),
                                    ctypes.c_int(batch), ctypes.c_float(lr), ctypes.c_uint64(seed), ctypes.byref(loss)))
        return loss.value
