"""C-ABI library on the CPU: it loads, exports every symbol include/hmat.h
declares, and its host-side tree builders agree bit-exactly with the oracle."""
import os
import re

import numpy as np
import pytest

import hmat_synth as hs
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hm():
    from paper_1703_09085_gb300 import build
    build.build()
    import paper_1703_09085_gb300 as g
    return g


class _NullCtx:
    h = None


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hmat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hmat_status|size_t|int64_t)\s+(\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(hm):
    decl = declared_symbols()
    assert len(decl) >= 20
    L = hm.lib()
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(hm.EXPORTS) == decl


@pytest.mark.parametrize("N,d,leaf", [(4, 2, 4), (64, 2, 32), (16, 3, 64), (13, 2, 8), (21, 3, 32), (32, 3, 64),
                                      (97, 2, 32), (128, 2, 32), (64, 3, 64)])
def test_trees_bit_exact_vs_oracle(hm, N, d, leaf):
    x = hs.grid_coords(N, d)
    ct = hm.ClusterTree(_NullCtx(), x, leaf)
    oc = oracle.ClusterTree(x, leaf)
    assert np.array_equal(ct.perm(), oc.perm())
    a, b = ct.nodes(), oc.nodes()
    for key in ("off", "size", "level", "parent", "nsons"):
        assert np.array_equal(a[key], b[key]), key
    bt = hm.BlockTree(_NullCtx(), ct, ct, 2.0)
    ob = oracle.BlockTree(oc, oc, 2.0)
    a, b = bt.nodes(), ob.nodes()
    for key in ("t", "s", "level", "parent", "kind"):
        assert np.array_equal(a[key], b[key]), key


def test_tree_edge_sizes(hm):
    # one point, and fewer points than a leaf: a single leaf cluster and one
    # dense block
    for x in (np.array([[0.5, 0.5]]), hs.grid_coords(3, 2)):
        ct = hm.ClusterTree(_NullCtx(), x, 16)
        assert np.array_equal(ct.perm(), np.arange(x.shape[0]))
        bt = hm.BlockTree(_NullCtx(), ct, ct, 2.0)
        nd = bt.nodes()
        assert len(nd["kind"]) == 1 and nd["kind"][0] == 1
    with pytest.raises(hm.HmatError):
        hm.ClusterTree(_NullCtx(), np.zeros((0, 2)), 16)  # no points


def test_tree_rejects_bad_input(hm):
    with pytest.raises(hm.HmatError):
        hm.ClusterTree(_NullCtx(), np.zeros((4, 2)), 1)  # duplicate points cannot be bisected
    with pytest.raises(hm.HmatError):
        hm.ClusterTree(_NullCtx(), np.zeros((4, 5)), 2)  # d must be 2 or 3


@pytest.mark.parametrize("name,nargs", [
    ("hmat_lu", 3), ("hmat_lu_batched", 4), ("hmat_invert", 3), ("hmat_cholesky", 3), ("hmat_addmul", 6),
    ("hmat_solve", 6), ("hmat_addeval", 7), ("trunc_lowrank", 10), ("hmat_create_from_csr", 7),
    ("hmat_clustertree_build", 6), ("hmat_blocktree_build", 5), ("hmat_copy_values", 3), ("hmat_to_dense", 3),
    ("hmat_stats_get", 2), ("hmat_ranks", 2), ("hmat_mlp_create", 3), ("hmat_lu_training_data", 5),
    ("hmat_analyze_lu", 7)])
def test_null_arguments_return_a_status(hm, name, nargs):
    """Every entry point checks its arguments on the host before touching a
    device: null arguments give HMAT_ERR_ARG and a message, never a crash."""
    import ctypes
    L = hm.lib()
    rc = getattr(L, name)(*([None] * nargs))
    assert rc == hm.HMAT_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    L.hmat_last_error(buf, ctypes.c_size_t(256))
    assert buf.value


def test_standard_schedule_builds_on_the_host(hm):
    """hmat_analyze_lu (host only) in both modes: the standard form applies
    every product at once (Section 4), so its schedule truncates more; a
    rank rule the mixed form cannot honour and an unknown mode are refused
    before any work."""
    import ctypes
    p = hs.small_laplace(16, 3, 64, 1e-4)
    ct = hm.ClusterTree(_NullCtx(), p.coords(), p.leaf)
    bt = hm.BlockTree(_NullCtx(), ct, ct, p.eta)
    csr = p.matrix()

    def analyze(mode, precision=hm.HMAT_FP64, rule=hm.HMAT_REL_FRO):
        o = hm.Opts(p.eps, 0, precision, 0, 0, None, 0, 0, mode, rule)
        st = hm.Stats()
        rc = hm.lib().hmat_analyze_lu(bt.h, ctypes.c_int64(csr.n),
                                      np.ascontiguousarray(csr.rowptr, np.int64).ctypes.data_as(hm.I64P),
                                      np.ascontiguousarray(csr.colidx, np.int64).ctypes.data_as(hm.I64P),
                                      np.ascontiguousarray(csr.val, np.float64).ctypes.data_as(hm.F64P),
                                      ctypes.byref(o), ctypes.byref(st))
        return rc, st.as_dict()

    rc_a, acc = analyze(hm.HMAT_ACCUMULATED)
    rc_s, std = analyze(hm.HMAT_STANDARD)
    assert rc_a == 0 and rc_s == 0
    # every product of a leaf pair is truncated into its target at once, so
    # the standard schedule holds more truncations (Section 4)
    assert std["truncations"] > acc["truncations"] > 0
    assert analyze(7)[0] == hm.HMAT_ERR_ARG
    assert analyze(hm.HMAT_ACCUMULATED, hm.HMAT_MIXED, hm.HMAT_REL_SPEC)[0] == hm.HMAT_ERR_ARG


def test_symbolic_pass_is_deterministic(hm):
    """The schedule of the 32^3 mixed H-LU (about a million tasks, so its level
    ordering runs on several host threads) comes out the same on every call."""
    import ctypes
    p = hs.laplace3d_32()
    ct = hm.ClusterTree(_NullCtx(), p.coords(), p.leaf)
    bt = hm.BlockTree(_NullCtx(), ct, ct, p.eta)
    csr = p.matrix()
    rp = np.ascontiguousarray(csr.rowptr, np.int64)
    ci = np.ascontiguousarray(csr.colidx, np.int64)
    va = np.ascontiguousarray(csr.val, np.float64)
    runs = []
    for _ in range(2):
        o = hm.Opts(p.eps, 0, hm.HMAT_MIXED, 0, 0, None, 0, 0, hm.HMAT_ACCUMULATED, hm.HMAT_REL_FRO)
        st = hm.Stats()
        assert hm.lib().hmat_analyze_lu(bt.h, ctypes.c_int64(csr.n), rp.ctypes.data_as(hm.I64P),
                                        ci.ctypes.data_as(hm.I64P), va.ctypes.data_as(hm.F64P), ctypes.byref(o),
                                        ctypes.byref(st)) == 0
        d = st.as_dict()
        runs.append(tuple(d[k] for k in ("tasks", "truncations", "levels", "critical_flops", "est_flops",
                                         "device_bytes")))
    assert runs[0] == runs[1]
    assert runs[0][0] > 500000
