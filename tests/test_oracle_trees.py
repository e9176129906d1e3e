"""Pins of the oracle's cluster and block trees (Section 2): a hand-derived
golden case and the defining properties on larger grids."""
import numpy as np
import pytest

import hmat_synth as hs
import oracle
from golden import read_tree


def test_golden_grid4x4():
    g = read_tree("tree_grid4x4_leaf4.txt")
    ct = oracle.ClusterTree(hs.grid_coords(4, 2), 4)
    assert list(ct.perm()) == g["perm"]
    cn = ct.nodes()
    got = [(i, int(cn["off"][i]), int(cn["size"][i]), int(cn["level"][i])) for i in range(len(cn["off"]))]
    assert got == [tuple(c) for c in g["clusters"]]
    bt = oracle.BlockTree(ct, ct, 2.0)
    bn = bt.nodes()
    got = [(int(bn["t"][b]), int(bn["s"][b]), int(bn["kind"][b])) for b in range(len(bn["t"]))]
    assert got == [tuple(b) for b in g["blocks"]]


def check_cluster_tree(ct, n, leaf):
    perm = ct.perm()
    assert sorted(perm) == list(range(n))
    cn = ct.nodes()
    sons = {i: [] for i in range(len(cn["off"]))}
    for i, p in enumerate(cn["parent"]):
        if p >= 0:
            sons[int(p)].append(i)
    assert cn["off"][0] == 0 and cn["size"][0] == n
    for i, ss in sons.items():
        if not ss:
            assert cn["size"][i] <= leaf
            continue
        # sons are disjoint and cover the father (Definition "Cluster tree")
        off = cn["off"][i]
        for s in ss:
            assert cn["off"][s] == off and cn["level"][s] == cn["level"][i] + 1
            off += cn["size"][s]
        assert off == cn["off"][i] + cn["size"][i]
        assert cn["size"][i] > leaf
    return cn, sons


@pytest.mark.parametrize("N,d,leaf", [(32, 2, 16), (9, 3, 16), (13, 2, 8)])
def test_tree_properties(N, d, leaf):
    n = N ** d
    ct = oracle.ClusterTree(hs.grid_coords(N, d), leaf)
    cn, csons = check_cluster_tree(ct, n, leaf)
    bt = oracle.BlockTree(ct, ct, 2.0)
    bn = bt.nodes()
    cover = np.zeros((n, n), np.int32)
    nb = len(bn["t"])
    bsons = {b: [] for b in range(nb)}
    for b, p in enumerate(bn["parent"]):
        if p >= 0:
            bsons[int(p)].append(b)
    for b in range(nb):
        t, s = int(bn["t"][b]), int(bn["s"][b])
        if bn["kind"][b] == 0:
            # sons(b) = sons(t) x sons(s)  (Definition "Block tree")
            pairs = sorted((int(bn["t"][c]), int(bn["s"][c])) for c in bsons[b])
            assert pairs == sorted((a, c) for a in csons[t] for c in csons[s])
            continue
        to, ts, so, ss = cn["off"][t], cn["size"][t], cn["off"][s], cn["size"][s]
        cover[to:to + ts, so:so + ss] += 1
        if bn["kind"][b] == 1:
            # admissible block tree: inadmissible leaf => t or s is a leaf
            assert not csons[t] or not csons[s]
    # leaves form a disjoint partition of I x I
    assert np.all(cover == 1)
    # diagonal blocks are never admissible
    for b in range(nb):
        if bn["t"][b] == bn["s"][b]:
            assert bn["kind"][b] != 2


def test_sparsity_constant_bounded():
    # C_sp: blocks per row cluster stays bounded as n grows (eq. blocktree_rowsparse)
    csp = []
    for N in (16, 32, 64):
        ct = oracle.ClusterTree(hs.grid_coords(N, 2), 16)
        bn = oracle.BlockTree(ct, ct, 2.0).nodes()
        csp.append(np.bincount(bn["t"]).max())
    assert csp[2] <= csp[1] + 2 and csp[2] < 40
