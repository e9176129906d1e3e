"""The stored oracle values of the full-size workloads
(tests/golden/oracle_<workload>.json) against the oracle as it is now, on the
CPU: the structural part (block-tree and permutation hashes, leaf counts) is
recomputed from the oracle's tree builders, and the stored numbers satisfy
what the method fixes (the rank histogram counts every admissible leaf, the
mean rank is the histogram's mean, the preconditioner error is of the order
of eps).  A stored file that no longer matches the oracle fails here before
any GPU test compares against it."""
import numpy as np
import pytest

import golden
import hmat_synth as hs
import oracle

WORKLOADS = {"laplace3d_32": hs.laplace3d_32, "laplace3d_64": hs.laplace3d_64}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_stored_structure_is_the_oracles(name):
    ref = golden.read_oracle_values(name)
    if ref is None:
        pytest.skip(f"no stored oracle values for {name}")
    p = WORKLOADS[name]()
    ct = oracle.ClusterTree(p.coords(), p.leaf)
    bt = oracle.BlockTree(ct, ct, p.eta)
    nodes = bt.nodes()
    assert (ref["n"], ref["leaf"], ref["eta"], ref["eps"]) == (p.n, p.leaf, p.eta, p.eps)
    assert ref["blocks"] == len(nodes["t"])
    assert ref["dense_leaves"] == int(np.sum(nodes["kind"] == 1))
    assert ref["lowrank_leaves"] == int(np.sum(nodes["kind"] == 2))
    assert ref["blocktree_sha256"] == golden.tree_hash(nodes)
    assert ref["perm_sha256"] == golden.perm_hash(ct.perm())


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_stored_numbers_are_consistent(name):
    ref = golden.read_oracle_values(name)
    if ref is None:
        pytest.skip(f"no stored oracle values for {name}")
    hist = np.asarray(ref["rank_histogram"])
    assert hist.sum() == ref["lowrank_leaves"]
    assert len(hist) == ref["max_rank"] + 1 and hist[-1] > 0
    assert abs((hist * np.arange(len(hist))).sum() / hist.sum() - ref["mean_rank"]) <= 1e-12 * ref["mean_rank"]
    # the factorisation truncates at least once per admissible leaf that ends
    # with a non-zero rank, and the preconditioner error is of the order of eps
    assert ref["truncations"] >= int(hist[1:].sum())
    assert 0.1 * ref["eps"] <= ref["precond_error"] <= 10.0 * ref["eps"]
    assert 1 <= ref["power_iterations"] <= 50
