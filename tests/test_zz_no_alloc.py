"""trunc_lowrank_noalloc: the truncation entry point that allocates no memory.

It exists for callers that cannot let the library allocate device memory: a
real-time host that reserves all device memory up front (an allocation in the
middle of a run could fail or stall) or an application whose own pool owns
the GPU.  Its scratch is a fixed array compiled into the library.  This file
is collected last on purpose: the first call on the device looks the array's
address up, and the test must pass both alone in a fresh process and after
every other test.
"""
import ctypes

import numpy as np
import pytest

import hmat_synth as hs
import oracle
from gpu_util import from_dev, hm, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_trunc_lowrank_on_two_calls_in_a_row():
    g = hm()
    ctx = g.Context(0)
    # two different problems back to back: the shared scratch must not carry
    # anything from the first call into the second
    for call, (m, n, ell, eps) in enumerate([(300, 200, 40, 1e-5), (64, 512, 70, 1e-4)]):
        A, B = hs.lowrank_stack(m, n, ell, seed=500 + call, decay=0.5)
        U1, V1 = to_dev(A), to_dev(B)
        k1 = g.trunc_lowrank(ctx, U1, V1, eps)
        U2, V2 = to_dev(A), to_dev(B)
        k2 = g.trunc_lowrank_noalloc(ctx, U2, V2, eps)
        assert k1 == k2 and k1 > 0
        P1 = from_dev(U1, k1) @ from_dev(V1, k1).T
        P2 = from_dev(U2, k2) @ from_dev(V2, k2).T
        nrm = np.linalg.norm(A @ B.T)
        assert np.linalg.norm(P1 - P2) <= 1e-11 * nrm
        # and both equal the oracle's truncation (Section 3, "Truncation")
        Co, Do = oracle.trunc(A, B, eps)
        assert Co.shape[1] == k2
        assert np.linalg.norm(P2 - Co @ Do.T) <= 1e-11 * nrm


def test_noalloc_rejects_problems_beyond_its_fixed_scratch():
    g = hm()
    ctx = g.Context(0)
    m, n, k = 200000, 200000, 16  # (2m + n) k doubles > the 2^21 - 32 available
    kn = ctypes.c_int64(-1)
    rc = g.lib().trunc_lowrank_noalloc(ctx.h, ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int64(k),
                                       ctypes.c_void_p(16), ctypes.c_int64(m), ctypes.c_void_p(16),
                                       ctypes.c_int64(n), ctypes.c_double(1e-4), ctypes.byref(kn))
    assert rc == 1  # HMAT_ERR_ARG, before any device work
    assert "exceeds the fixed scratch" in g.last_error()
    assert kn.value == -1
    # a NaN tolerance and leading dimensions beyond 32 bits are refused the same way
    for eps, ld in ((float("nan"), 100), (1e-4, 2**31)):
        rc = g.lib().trunc_lowrank_noalloc(ctx.h, ctypes.c_int64(100), ctypes.c_int64(100), ctypes.c_int64(4),
                                           ctypes.c_void_p(16), ctypes.c_int64(ld), ctypes.c_void_p(16),
                                           ctypes.c_int64(100), ctypes.c_double(eps), ctypes.byref(kn))
        assert rc == 1 and kn.value == -1
